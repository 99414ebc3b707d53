"""Differentiation through the solve (GPU): torch.autograd.Function with an adjoint-solve backward.

Configuration 5 of the build: 3D convection-diffusion with learnable per-axis Peclet
numbers (3 FP64 scalars), s = 16 Gaussian right-hand sides, loss ||X - X*||_F^2 with a
seeded target; forward eGl-BiCG (Algorithm 4), backward A^H Lambda = dL/dX with the same
method.  Checked against a dense-solve reference gradient and central finite differences
(h = 1e-6) on a 12^3 copy, and against finite differences of GPU solves on 64^3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import ConvDiff, convdiff_csr, gaussian_block  # noqa: E402
from workloads.stencil import convdiff_dpe_csr  # noqa: E402

pytestmark = pytest.mark.gpu

PE0 = (0.3, 0.2, 0.1)
SHIFT = 0.05j


@pytest.fixture(scope="module")
def kr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as m
    m.load_library()
    return m


def setup(N, s=16):
    op = ConvDiff((N, N, N), (0.0, 0.0, 0.0), SHIFT)
    rp, ci, base = convdiff_csr(op)
    d = [convdiff_dpe_csr(op, a).real for a in range(3)]
    B = gaussian_block(op.n, s, seed=0)
    Xs = gaussian_block(op.n, s, seed=1) * 0.1
    return op, rp, ci, base, d, B, Xs


def vals_of(base, d, pe):
    return base + sum(pe[a] * d[a] for a in range(3))


def dense_loss_and_grad(n, rp, ci, base, d, pe, B, Xs):
    import scipy.sparse as sp
    v = vals_of(base, d, pe)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    X = np.linalg.solve(A, B)
    L = float(np.sum(np.abs(X - Xs) ** 2))
    G = 2 * (X - Xs)                       # dL/dRe X + i dL/dIm X
    Lam = np.linalg.solve(A.conj().T, G)   # adjoint solve
    rows = np.repeat(np.arange(n), np.diff(rp))
    gv = -np.sum(Lam[rows] * np.conj(X[ci]), axis=1)   # dL/dA_ij on the pattern
    gpe = np.array([float(np.real(np.sum(gv * d[a]))) for a in range(3)])
    return L, gpe, Lam


def gpu_loss_and_grad(kr, op_h, base_t, d_t, pe, B_t, Xs_t, tol, method="egl_bicg"):
    from paper_1504_04395_gb300.autograd import krylov_solve
    pe_t = torch.tensor(pe, dtype=torch.float64, device="cuda", requires_grad=True)
    B_req = B_t.clone().requires_grad_(True)
    vals = base_t + pe_t[0] * d_t[0] + pe_t[1] * d_t[1] + pe_t[2] * d_t[2]
    X = krylov_solve(vals, B_req, op_h, method, tol, 4000)
    L = torch.sum(torch.abs(X - Xs_t) ** 2)
    L.backward()
    return float(L.item()), pe_t.grad.cpu().numpy(), B_req.grad


def test_gradient_12cube_dense_and_fd(kr):
    op, rp, ci, base, d, B, Xs = setup(12)
    n = op.n
    L_ref, g_ref, Lam_ref = dense_loss_and_grad(n, rp, ci, base, d, PE0, B, Xs)
    # central finite differences with dense solves (h = 1e-6)
    h = 1e-6
    g_fd = np.zeros(3)
    for a in range(3):
        pp = list(PE0); pm = list(PE0)
        pp[a] += h; pm[a] -= h
        g_fd[a] = (dense_loss_and_grad(n, rp, ci, base, d, pp, B, Xs)[0]
                   - dense_loss_and_grad(n, rp, ci, base, d, pm, B, Xs)[0]) / (2 * h)
    assert np.allclose(g_fd, g_ref, rtol=1e-6, atol=0)
    # GPU autograd (forward eGl-BiCG, backward adjoint eGl-BiCG)
    op_h = kr.Operator(n, rp, ci, vals_of(base, d, PE0))
    base_t = torch.from_numpy(base).cuda()
    d_t = [torch.from_numpy(x).cuda() for x in d]
    L, g, gB = gpu_loss_and_grad(kr, op_h, base_t, d_t, PE0, torch.from_numpy(B).cuda(),
                                 torch.from_numpy(Xs).cuda(), tol=1e-8)
    assert abs(L - L_ref) / L_ref < 1e-7
    assert np.allclose(g, g_ref, rtol=1e-6, atol=0), (g, g_ref)
    assert np.linalg.norm(gB.cpu().numpy() - Lam_ref) / np.linalg.norm(Lam_ref) < 1e-6
    op_h.close()


@pytest.mark.parametrize("method", ["gl_bicg", "bl_bicg"])
def test_gradient_other_methods_12cube(kr, method):
    op, rp, ci, base, d, B, Xs = setup(12, s=4)
    n = op.n
    _, g_ref, _ = dense_loss_and_grad(n, rp, ci, base, d, PE0, B, Xs)
    op_h = kr.Operator(n, rp, ci, vals_of(base, d, PE0))
    _, g, _ = gpu_loss_and_grad(kr, op_h, torch.from_numpy(base).cuda(), [torch.from_numpy(x).cuda() for x in d],
                                PE0, torch.from_numpy(B).cuda(), torch.from_numpy(Xs).cuda(), tol=1e-10,
                                method=method)
    assert np.allclose(g, g_ref, rtol=1e-6, atol=0), (g, g_ref)
    op_h.close()


def test_gradient_64cube_fd(kr):
    """Full configuration (64^3, n = 262144, s = 16): autograd gradient vs central FD of GPU solves."""
    op, rp, ci, base, d, B, Xs = setup(64)
    n = op.n
    op_h = kr.Operator(n, rp, ci, vals_of(base, d, PE0))
    base_t = torch.from_numpy(base).cuda()
    d_t = [torch.from_numpy(x).cuda() for x in d]
    B_t = torch.from_numpy(B).cuda()
    Xs_t = torch.from_numpy(Xs).cuda()
    L, g, gB = gpu_loss_and_grad(kr, op_h, base_t, d_t, PE0, B_t, Xs_t, tol=1e-8)
    assert gB.shape == (n, 16) and torch.isfinite(gB.abs()).all()

    def loss(pe):
        v = vals_of(base, d, pe)
        kr.kr_op_update_values(op_h, v)
        X, info = kr.kr_solve(op_h, "egl_bicg", B_t, tol=1e-13, maxit=4000)
        assert info.relres_true < 1e-12
        return float(torch.sum(torch.abs(X - Xs_t) ** 2).item())

    h = 1e-6
    for a in range(3):
        pp = list(PE0); pm = list(PE0)
        pp[a] += h; pm[a] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - g[a]) <= 1e-4 * np.max(np.abs(g)), (a, fd, g[a])
    op_h.close()
