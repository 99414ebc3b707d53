"""Matrix-free 4D lattice operator (GPU) against the oracle's sparse product.

`kr_op_create_lattice4d` applies the Wilson-type operator of Example 4 from its links and
gamma matrices (spin projection before the link multiply); the oracle multiplies by the
assembled 49-entries-per-row sparse matrix of the same lattice (`workloads.lattice_csr`).
Products (A and A^H, complex128 and complex64) are compared element by element with
bounds from the error analysis of a sum of products, fused reductions to the usual
bounds, and whole solves against the CSR operator and the oracle's residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import Lattice4D, gaussian_block, lattice_csr  # noqa: E402
from workloads.lattice import GAMMA, LATTICE_MASS, haar_links  # noqa: E402

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def kr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as m
    m.load_library()
    yield m
    m.kr_set_lattice_rows_per_thread(0)


@pytest.fixture(params=[4, 12], ids=["rows4", "rows12"])
def variant(kr, request):
    """Both kernels of the matrix-free product: (site, colour) units and whole sites."""
    kr.kr_set_lattice_rows_per_thread(request.param)
    yield request.param
    kr.kr_set_lattice_rows_per_thread(0)


def make(kr, dims, seed=0, links=None):
    L = Lattice4D(dims, LATTICE_MASS, seed=seed)
    U = haar_links(dims, seed) if links is None else links
    rp, ci, v = lattice_csr(L, U)
    op = kr.Operator.lattice4d(dims, 4.0 + LATTICE_MASS, -0.5, GAMMA, U)
    return L, U, rp, ci, v, op


def dev(x, dtype=np.complex128):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).astype(dtype))).cuda()


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("dims", [(3, 4, 5, 3), (6, 6, 6, 6)])
@pytest.mark.parametrize("s", [1, 3, 8, 12, 32])
def test_lattice_product_fp64(kr, variant, dims, s):
    L, U, rp, ci, v, op = make(kr, dims)
    assert op.info()["nnz"] == 49 * L.n
    A = oracle.csr_matrix_from_arrays(L.n, rp, ci, v)
    V = gaussian_block(L.n, s, seed=s)
    for adj in (False, True):
        M = oracle.adjoint(A) if adj else A
        Y = kr.kr_op_apply(op, dev(V), adjoint=adj).cpu().numpy()
        ref = oracle.spmm(M, V)
        scale = abs(M) @ np.abs(V)
        # 49 terms per entry, regrouped by the spin projection: a few ulps per term
        assert np.all(np.abs(Y - ref) <= 64 * 49 * U64 * scale), (dims, s, adj)
    op.close()


@pytest.mark.parametrize("s", [1, 2, 8, 32])
def test_lattice_product_c64(kr, variant, s):
    dims = (4, 3, 5, 4)
    L, U, rp, ci, v, op = make(kr, dims)
    # the complex64 kernel uses the links rounded to complex64 (times the exact hop -1/2);
    # the CSR entries (+-1/2, +-i/2) x U round the same way
    A = oracle.csr_matrix_from_arrays(L.n, rp, ci, c64(v))
    V = c64(gaussian_block(L.n, s, seed=s))
    for adj in (False, True):
        M = oracle.adjoint(A) if adj else A
        Y, _ = kr.kr_op_apply_reduce_c64(op, dev(V, np.complex64), adjoint=adj)
        ref = oracle.spmm(M, V)
        scale = abs(M) @ np.abs(V)
        err = np.abs(Y.cpu().numpy().astype(np.complex128) - ref)
        assert np.all(err <= 8 * 49 * U32 * scale + 1e-30), (s, adj)
    op.close()


@pytest.mark.parametrize("s", [4, 12])
@pytest.mark.parametrize("kind", ["gram", "trace", "sumv", "norm2"])
def test_lattice_fused_reductions(kr, variant, s, kind):
    L, U, rp, ci, v, op = make(kr, (4, 4, 4, 5))
    A = oracle.csr_matrix_from_arrays(L.n, rp, ci, v)
    V = gaussian_block(L.n, s, seed=1)
    Um = gaussian_block(L.n, s, seed=2) if kind != "sumv" else gaussian_block(L.n, 1, seed=2)[:, 0].copy()
    Ud = dev(Um) if kind != "norm2" else None
    Y, out = kr.kr_op_apply_reduce(op, dev(V), Ud, kind=kind)
    Yr = A @ V
    if kind == "gram":
        ref = oracle.gram(Um, Yr)
        bound = (np.abs(Um).T @ np.abs(Yr)).sum()
    elif kind == "trace":
        ref = np.array([oracle.trace_ip(Um, Yr)])
        bound = (np.abs(Um) * np.abs(Yr)).sum()
    elif kind == "sumv":
        ref = np.array([oracle.sum_ip(Um, Yr)])
        bound = (np.abs(Um)[:, None] * np.abs(Yr)).sum()
    else:
        ref = np.array([np.linalg.norm(Yr) ** 2])
        bound = ref.real.sum()
    got = out.cpu().numpy().reshape(ref.shape)
    if kind == "norm2":
        got = got.real
    assert np.max(np.abs(got - ref)) <= 1e-12 * bound
    _, out2 = kr.kr_op_apply_reduce(op, dev(V), Ud, kind=kind)
    assert torch.equal(out, out2)  # fixed summation order
    op.close()


@pytest.mark.parametrize("method", ["egl_bicg", "bl_bicgstab", "gl_qmr", "bl_bicg_rq"])
def test_lattice_operator_solves(kr, variant, method):
    """Solves with the matrix-free operator reach the tolerance on the oracle's sparse matrix and
    agree with the CSR operator's solution."""
    dims = (6, 6, 6, 6)
    L, U, rp, ci, v, op = make(kr, dims)
    csr = kr.Operator(L.n, rp, ci, v)
    A = oracle.csr_matrix_from_arrays(L.n, rp, ci, v)
    B = gaussian_block(L.n, 12, seed=12)
    X1, i1 = kr.kr_solve(op, method, dev(B), tol=1e-10, maxit=2000)
    X2, i2 = kr.kr_solve(csr, method, dev(B), tol=1e-10, maxit=2000)
    assert i1.status == "OK" and i2.status == "OK", (i1, i2)
    X1 = X1.cpu().numpy()
    X2 = X2.cpu().numpy()
    assert np.linalg.norm(B - A @ X1) / np.linalg.norm(B) < 2e-10
    assert np.linalg.norm(X1 - X2) / np.linalg.norm(X2) < 1e-8
    assert abs(i1.iters - i2.iters) <= max(3, i2.iters // 10)
    op.close()
    csr.close()


def test_lattice_first_iterations_match_oracle(kr):
    """eGl-BiCG on the matrix-free operator: the first 20 residual norms against the oracle's
    run on the sparse matrix (global and economic methods are insensitive at this level)."""
    dims = (6, 6, 6, 6)
    L, U, rp, ci, v, op = make(kr, dims)
    A = oracle.csr_matrix_from_arrays(L.n, rp, ci, v)
    B = gaussian_block(L.n, 12, seed=3)
    ref = oracle.solve("egl_bicg", A, B, tol=1e-12, maxit=20)
    X, info = kr.kr_solve(op, "egl_bicg", dev(B), tol=1e-12, maxit=20, check_every=1)
    h = np.array(info.history[:21])
    r = np.array(ref.history[:21])
    assert np.all(np.abs(h - r) <= 1e-10 * r), np.max(np.abs(h - r) / r)
    op.close()


def test_lattice_mixed_precision(kr):
    """Complex64 inner solves on the matrix-free operator inside FP64 defect correction."""
    dims = (6, 6, 6, 6)
    L, U, rp, ci, v, op = make(kr, dims)
    A = oracle.csr_matrix_from_arrays(L.n, rp, ci, v)
    B = gaussian_block(L.n, 32, seed=32)
    X, info = kr.kr_solve(op, "egl_bicg", dev(B), tol=1e-10, maxit=3000, precision=kr.FP32_REFINE)
    assert info.status == "OK" and info.outer_iters >= 2 and info.fp64_iters == 0, info
    X = X.cpu().numpy()
    assert np.linalg.norm(B - A @ X) / np.linalg.norm(B) <= 1.01e-10
    op.close()


def test_lattice_operator_rejects_unsupported_calls(kr):
    L, U, rp, ci, v, op = make(kr, (3, 3, 3, 3))
    with pytest.raises(kr.KrylovError):
        kr.kr_op_update_values(op, v)
    op.close()


def _lattice_rows_by_definition(dims, diag, hop, links, V_nb, sites_idx, spins, colours):
    """Rows (x, a, c) of A V from the operator's definition, entry by entry:
    y = d v_x + hop sum_mu [ (I - gamma_mu) (x) U_mu(x) v_{x+mu} + (I + gamma_mu) (x) U_mu(x-mu)^H v_{x-mu} ].
    V_nb(x) returns the (4, 3, s) block of V at site x."""
    strides = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    eye = np.eye(4)
    out = []
    for x, a, c in zip(sites_idx, spins, colours):
        coords, rem = [], x
        for L in dims:
            coords.append(rem % L)
            rem //= L
        y = diag * V_nb(x)[a, c]
        for mu in range(4):
            fw = x + (((coords[mu] + 1) % dims[mu]) - coords[mu]) * strides[mu]
            bw = x + (((coords[mu] - 1) % dims[mu]) - coords[mu]) * strides[mu]
            Pf = eye - GAMMA[mu]
            Pb = eye + GAMMA[mu]
            Vf, Vb = V_nb(fw), V_nb(bw)
            for b in range(4):
                for cp in range(3):
                    y = y + hop * Pf[a, b] * links[mu, x, c, cp] * Vf[b, cp]
                    y = y + hop * Pb[a, b] * np.conj(links[mu, bw, cp, c]) * Vb[b, cp]
        out.append(y)
    return np.array(out)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_lattice_full_size_sampled_rows(kr, dtype):
    """Config-4 size (24^4 x 12, n = 3,981,312), s = 32, the launch the mixed-precision bench
    times: 400 sampled rows (and the first and last) recomputed from the operator's definition."""
    dims = (24, 24, 24, 24)
    sites = 24 ** 4
    n = 12 * sites
    s = 32
    U = haar_links(dims, 0)
    op = kr.Operator.lattice4d(dims, 4.0 + LATTICE_MASS, -0.5, GAMMA, U)
    g = torch.Generator(device="cuda").manual_seed(7)
    V = torch.complex(torch.randn(n, s, device="cuda", generator=g, dtype=torch.float64),
                      torch.randn(n, s, device="cuda", generator=g, dtype=torch.float64))
    if dtype == "c64":
        V32 = V.to(torch.complex64)
        Y, _ = kr.kr_op_apply_reduce_c64(op, V32)
        V = V32.to(torch.complex128)
        Uref = c64(U * -0.5) / -0.5  # the kernel multiplies by the hop-scaled links rounded to complex64
    else:
        Y = kr.kr_op_apply(op, V)
        Uref = U
    rng = np.random.default_rng(24)
    rows = np.concatenate([rng.integers(0, n, 400), [0, n - 1]])
    xs, rem = rows // 12, rows % 12
    a_s, c_s = rem // 3, rem % 3
    Vsite = V.view(sites, 4, 3, s)

    cache = {}

    def V_nb(x):
        if x not in cache:
            cache[x] = Vsite[int(x)].cpu().numpy()
        return cache[x]

    ref = _lattice_rows_by_definition(dims, 4.0 + LATTICE_MASS, -0.5, Uref, V_nb, xs, a_s, c_s)
    got = Y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
    # scale: a bound on the sum of |terms| per entry (diagonal 2.2 |v|, 48 hop terms <= |v| / 2)
    scale = 50 * float(V.abs().max())
    u = U32 if dtype == "c64" else U64
    assert np.all(np.abs(got - ref) <= 64 * u * scale), np.max(np.abs(got - ref) / scale)
    op.close()
