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
