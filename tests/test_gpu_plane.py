"""Complex64 stencil product marching grid planes through shared memory (GPU).

For the matrix-free (2d+1)-point stencil on a 2D or 3D grid the complex64 product runs on the
plane kernel (TMA tensor copies of each x-y tile's plane with its halo; see
kr_plane_c64.cuh).  Its product is compared bit for bit with the products of the stored CSR
matrix of the same stencil (every kernel applies the entries in the same order), and its fused
reductions with FP64 sums on the host of the complex64 inputs, within the bound of the standard
error analysis of FP32 sums.  Grids whose extents are not multiples of the tile (ragged tiles
in x and y), 2D grids (one plane), a 1D grid (which the plane kernel does not take), every
supported s and both A and A^H.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import ConvDiff, convdiff_csr, gaussian_block  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as m
    m.load_library()
    m.kr_take_device_timeouts(reset=True)
    yield m
    m.kr_set_tile_kernels(True)
    m.kr_set_column_pairs(True)


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def dev32(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).astype(np.complex64))).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def pair(kr, dims, shift=0.05j):
    cd = ConvDiff(dims, tuple([0.4, -0.3, 0.2][: len(dims)]), shift)
    rp, ci, v = convdiff_csr(cd)
    centre, minus, plus = cd.coefficients()
    st = kr.Operator.stencil(dims, centre, minus, plus)
    csr = kr.Operator(cd.n, rp, ci, v)
    return cd, st, csr, oracle.csr_matrix_from_arrays(cd.n, rp, ci, c64(v))


@pytest.mark.parametrize("dims", [(37, 11, 9), (70, 13, 5), (33, 17), (64, 64), (41,)])
@pytest.mark.parametrize("s", [2, 4, 8, 16, 32])
def test_plane_product_equals_csr(kr, dims, s):
    cd, st, csr, A = pair(kr, dims)
    V = c64(gaussian_block(cd.n, s, seed=s))
    Vd = dev32(V)
    for adj in (False, True):
        Ys, _ = kr.kr_op_apply_reduce_c64(st, Vd, adjoint=adj)
        kr.kr_set_tile_kernels(False)
        try:
            Yc, _ = kr.kr_op_apply_reduce_c64(csr, Vd, adjoint=adj)
        finally:
            kr.kr_set_tile_kernels(True)
        assert torch.equal(Ys, Yc), (dims, s, adj)
        M = oracle.adjoint(A) if adj else A
        ref = oracle.spmm(M, V)
        scale = abs(M) @ np.abs(V)
        assert np.all(np.abs(host(Ys) - ref) <= 4 * 9 * 2.0 ** -24 * scale + 1e-30)
    st.close()
    csr.close()


@pytest.mark.parametrize("dims", [(37, 11, 9), (33, 17)])
@pytest.mark.parametrize("s", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("kind", ["gram", "trace", "sumv", "norm2"])
def test_plane_fused_reductions(kr, dims, s, kind):
    cd, st, csr, A = pair(kr, dims)
    V = c64(gaussian_block(cd.n, s, seed=3))
    U = c64(gaussian_block(cd.n, s, seed=4) if kind != "sumv" else gaussian_block(cd.n, 1, seed=4)[:, 0])
    Ud = dev32(U) if kind != "norm2" else None
    Y, out = kr.kr_op_apply_reduce_c64(st, dev32(V), Ud, kind=kind)
    Yk = host(Y)
    assert np.max(np.abs(Yk - oracle.spmm(A, V)) / (abs(A) @ np.abs(V))) < 4 * 9 * 2.0 ** -24
    if kind == "gram":
        ref, bound = U.conj().T @ Yk, np.abs(U).T @ np.abs(Yk)
    elif kind == "trace":
        ref, bound = np.array([np.sum(U.conj() * Yk)]), np.array([np.sum(np.abs(U) * np.abs(Yk))])
    elif kind == "sumv":
        ref = np.array([np.sum(U.conj()[:, None] * Yk)])
        bound = np.array([np.sum(np.abs(U)[:, None] * np.abs(Yk))])
    else:
        ref = np.array([np.linalg.norm(Yk) ** 2])
        bound = ref.copy()
    got = host(out).reshape(ref.shape)
    if kind == "norm2":
        got = got.real
    assert np.all(np.abs(got - ref) <= 1e-4 * bound), (kind, s)
    # the fixed summation order: bitwise reproducible
    _, out2 = kr.kr_op_apply_reduce_c64(st, dev32(V), Ud, kind=kind)
    assert torch.equal(out, out2)
    st.close()
    csr.close()


@pytest.mark.parametrize("s", [8, 16])
def test_plane_full_size_gram(kr, s):
    """128^3 (the benchmark's grid), fused Gram U^H (A V): the product on 2004 sampled rows and the
    Gram against FP64 on the host from the CSR matrix's product."""
    cd, st, csr, A = pair(kr, (128, 128, 128), shift=0.05j)
    V = c64(gaussian_block(cd.n, s, seed=1))
    U = c64(gaussian_block(cd.n, s, seed=2))
    Y, G = kr.kr_op_apply_reduce_c64(st, dev32(V), dev32(U), kind="gram")
    Yk = host(Y)
    rows = np.random.default_rng(0).choice(cd.n, 2004, replace=False)
    Ar = A[rows]
    ref = Ar @ V
    assert np.max(np.abs(Yk[rows] - ref) / (abs(Ar) @ np.abs(V))) < 4 * 9 * 2.0 ** -24
    Gh = U.conj().T @ Yk
    bound = np.abs(U).T @ np.abs(Yk)
    assert np.all(np.abs(host(G) - Gh) <= 1e-4 * bound)
    st.close()
    csr.close()


def test_plane_mixed_solve(kr):
    """Mixed-precision eGl-BiCG on the matrix-free stencil (its complex64 products on the plane
    kernel) reaches the FP64 tolerance, with the same iterations as the CSR storage's solve."""
    cd, st, csr, A = pair(kr, (24, 24, 24), shift=0.05j)
    B = gaussian_block(cd.n, 8, seed=5)
    Xs, infos = kr.kr_solve(st, "egl_bicg", torch.from_numpy(B).cuda(), tol=1e-10, maxit=2000,
                            precision=kr.FP32_REFINE)
    assert infos.status == "OK", infos
    Ah = oracle.csr_matrix_from_arrays(cd.n, *convdiff_csr(cd))
    res = np.linalg.norm(B - Ah @ Xs.cpu().numpy()) / np.linalg.norm(B)
    assert res <= 1.01e-10
    st.close()
    csr.close()


def test_plane_no_device_wait_ran_out(kr):
    assert kr.kr_take_device_timeouts(reset=False) == 0
