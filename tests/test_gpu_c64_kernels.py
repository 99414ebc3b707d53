"""Complex64 kernels of the mixed-precision inner solves (GPU).

The block product A V / A^H V and the fused reductions of Algorithms 2-5 in
complex64, called through kr_op_apply_reduce_c64 and kr_block_reduce_c64, are
compared with the FP64 oracle evaluated on the complex64 inputs (A, V, U rounded
to complex64 and widened back, so the only differences are the kernels' FP32
roundings), with bounds from the standard error analysis of a sum of products.

All three complex64 product kernels are covered: the row-tile kernel whose tiles are
staged in shared memory by bulk asynchronous copies (kr_set_tile_kernels), two adjacent
columns per thread (kr_set_column_pairs), and one column per thread.  They compute
every output entry with the same operations in the same order, so their products are
compared bit for bit; their reductions group the partial sums differently and agree to
FP32 rounding.  After the tests no bounded device wait of the tile kernel has run out.
"""
import numpy as np
import pytest
from scipy.sparse.linalg import splu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import ConvDiff, convdiff_csr, gaussian_block, random_csr  # noqa: E402

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24  # unit roundoff of FP32


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
    m.kr_set_column_pairs(True)
    m.kr_set_tile_kernels(True)


def c64(x):
    """Round to complex64 and widen back (the values the complex64 kernels see)."""
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def dev32(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).astype(np.complex64))).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def with_pairs(kr, on, fn):
    """on: True = column pairs (tile kernel off), False = one column (tile kernel off), "tile" = default."""
    kr.kr_set_tile_kernels(on == "tile")
    kr.kr_set_column_pairs(on is not False)
    try:
        return fn()
    finally:
        kr.kr_set_column_pairs(True)
        kr.kr_set_tile_kernels(True)


VARIANTS = ("tile", True, False)


SIZES = [1, 7, 1000, 5003]
S_VALUES = [1, 2, 3, 4, 6, 8, 16, 17, 32]


@pytest.mark.parametrize("real_offdiag", [False, True])
@pytest.mark.parametrize("s", S_VALUES)
def test_c64_spmm_matches_oracle(kr, s, real_offdiag):
    for n in SIZES:
        rp, ci, v = random_csr(n, seed=n + s, real_offdiag=real_offdiag)
        A = oracle.csr_matrix_from_arrays(n, rp, ci, c64(v))
        op = kr.Operator(n, rp, ci, v)
        V = c64(gaussian_block(n, s, seed=3))
        Vd = dev32(V)
        kmax = int(np.max(np.diff(rp))) if n else 0
        for adj in (False, True):
            M = oracle.adjoint(A) if adj else A
            ref = oracle.spmm(M, V)
            scale = abs(M) @ np.abs(V)
            outs = []
            for pairs in VARIANTS:
                Y, _ = with_pairs(kr, pairs, lambda: kr.kr_op_apply_reduce_c64(op, Vd, adjoint=adj))
                outs.append(Y)
                # each entry: at most kmax + 1 complex products summed in FP32
                err = np.abs(host(Y) - ref)
                assert np.all(err <= 4 * (kmax + 2) * U32 * scale + 1e-30), (n, s, adj, pairs)
            assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2]), (n, s, adj)
        op.close()


@pytest.mark.parametrize("s", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("kind", ["gram", "trace", "sumv", "norm2"])
def test_c64_fused_reductions(kr, s, kind):
    n = 6007
    rp, ci, v = random_csr(n, seed=s)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, c64(v))
    op = kr.Operator(n, rp, ci, v)
    V = c64(gaussian_block(n, s, seed=1))
    U = c64(gaussian_block(n, s, seed=2) if kind != "sumv" else gaussian_block(n, 1, seed=2)[:, 0])
    Ud = dev32(U) if kind != "norm2" else None
    res = {}
    # the per-thread kernels hold a fused s x s Gram in registers for s <= 16 only
    variants = ("tile",) if (kind == "gram" and s > 16) else VARIANTS
    for pairs in variants:
        res[pairs] = with_pairs(kr, pairs, lambda: kr.kr_op_apply_reduce_c64(op, dev32(V), Ud, kind=kind))
    for pairs in variants[1:]:
        assert torch.equal(res["tile"][0], res[pairs][0])
    res.setdefault(True, res["tile"])
    Yk = host(res[True][0])  # the stored complex64 product
    if kind == "gram":
        ref = oracle.gram(U, Yk)
        bound = np.abs(U).T @ np.abs(Yk)
    elif kind == "trace":
        ref = np.array([oracle.trace_ip(U, Yk)])
        bound = np.array([(np.abs(U) * np.abs(Yk)).sum()])
    elif kind == "sumv":
        ref = np.array([oracle.sum_ip(U, Yk)])
        bound = np.array([(np.abs(U)[:, None] * np.abs(Yk)).sum()])
    else:
        ref = np.array([np.linalg.norm(Yk) ** 2])
        bound = ref.copy()
    for pairs in variants:
        got = host(res[pairs][1]).reshape(ref.shape)
        if kind == "norm2":
            got = got.real
        # FP32 partial sums of at most a few hundred terms per thread, then FP64
        assert np.all(np.abs(got - ref) <= 1e-4 * bound.reshape(ref.shape)), (kind, pairs)
    # the stand-alone complex64 reduction of the stored product agrees to FP32 rounding
    for pairs in (True, False) if not (kind == "gram" and s > 16) else ():
        out2 = with_pairs(kr, pairs, lambda: kr.kr_block_reduce_c64(Ud, res[True][0], kind=kind))
        got2 = host(out2).reshape(ref.shape)
        if kind == "norm2":
            got2 = got2.real
        assert np.all(np.abs(got2 - ref) <= 1e-4 * bound.reshape(ref.shape)), (kind, pairs)
    # fixed summation order: bitwise reproducible
    _, out3 = kr.kr_op_apply_reduce_c64(op, dev32(V), Ud, kind=kind)
    assert torch.equal(out3, res["tile"][1])
    op.close()


@pytest.mark.parametrize("dims", [(9, 7, 13), (40, 33, 17)])
@pytest.mark.parametrize("s", [2, 8, 32])
def test_c64_stencil_equals_csr(kr, dims, s):
    """Matrix-free and CSR complex64 products: same entries in the same order, bitwise."""
    cd = ConvDiff(dims, (0.4, -0.3, 0.2), 0.05j)
    rp, ci, v = convdiff_csr(cd)
    centre, minus, plus = cd.coefficients()
    st = kr.Operator.stencil(dims, centre, minus, plus)
    csr = kr.Operator(cd.n, rp, ci, v)
    Vd = dev32(gaussian_block(cd.n, s, seed=s))
    for pairs in VARIANTS:
        for adj in (False, True):
            Ys, _ = with_pairs(kr, pairs, lambda: kr.kr_op_apply_reduce_c64(st, Vd, adjoint=adj))
            Yc, _ = with_pairs(kr, pairs, lambda: kr.kr_op_apply_reduce_c64(csr, Vd, adjoint=adj))
            assert torch.equal(Ys, Yc), (dims, s, adj, pairs)
    st.close()
    csr.close()


@pytest.mark.parametrize("method", ["gl_bicg", "egl_bicg", "li_bicg", "gl_bicgstab", "li_bicgstab", "egl_qmr",
                                    "li_qmr"])
def test_mixed_solve_with_and_without_pairs(kr, method):
    """FP64 defect correction over complex64 inner solves converges to the FP64 tolerance on
    both complex64 kernel variants, to the solution of a direct sparse LU."""
    cd = ConvDiff((24, 24, 24), (0.6, 0.6, 0.6), 0.05j)
    rp, ci, v = convdiff_csr(cd)
    op = kr.Operator(cd.n, rp, ci, v)
    s = 8
    B = gaussian_block(cd.n, s, seed=7)
    A = oracle.csr_matrix_from_arrays(cd.n, rp, ci, v)
    X_lu = splu(A.tocsc()).solve(B)  # direct sparse LU: the exact solution to rounding
    for pairs in VARIANTS:
        X, info = with_pairs(kr, pairs, lambda: kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10,
                                                            maxit=2000, precision=kr.FP32_REFINE))
        assert info.status == "OK", (method, pairs, info)
        X = host(X)
        res = np.linalg.norm(B - A @ X) / np.linalg.norm(B)
        assert res <= 1.01e-10, (method, pairs, res)
        assert np.linalg.norm(X - X_lu) / np.linalg.norm(X_lu) < 1e-8
        assert info.fp64_iters == 0, (method, pairs, info)
    op.close()


@pytest.mark.parametrize("method", ["bl_bicg_rq", "bl_bicgstab"])
def test_mixed_block_methods(kr, method):
    """Block methods under the defect correction.  With its s x s Gram products accumulated in
    FP32, the complex64 inner Bl-BiCG-rQ solve on this problem can stop reducing the residual,
    depending on how the partial sums are grouped (an oracle Bl-BiCG run with only its Grams
    rounded to FP32 diverges); the defect correction then restores X and finishes with the FP64
    solver.  Either way the result meets the FP64 tolerance."""
    cd = ConvDiff((24, 24, 24), (0.6, 0.6, 0.6), 0.05j)
    rp, ci, v = convdiff_csr(cd)
    op = kr.Operator(cd.n, rp, ci, v)
    B = gaussian_block(cd.n, 8, seed=7)
    A = oracle.csr_matrix_from_arrays(cd.n, rp, ci, v)
    X_lu = splu(A.tocsc()).solve(B)
    X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10, maxit=3000,
                          precision=kr.FP32_REFINE)
    assert info.status == "OK", info
    assert info.iters < 3000
    X = host(X)
    assert np.linalg.norm(B - A @ X) / np.linalg.norm(B) <= 1.01e-10
    assert np.linalg.norm(X - X_lu) / np.linalg.norm(X_lu) < 1e-8
    op.close()


@pytest.mark.parametrize("method", ["egl_bicg", "bl_bicg_rq"])
def test_mixed_fallback_to_fp64(kr, method):
    """The defect correction's FP64 finish: with every entry of A scaled by 2^130 (exact in FP64,
    beyond the complex64 range) the complex64 inner solve returns no finite correction, so the
    first defect-correction step does not reduce the residual; X is restored and the FP64 solver
    finishes to the requested tolerance.  The solution is 2^-130 times that of the unscaled system."""
    cd = ConvDiff((16, 16, 16), (0.6, 0.6, 0.6), 0.05j)
    rp, ci, v = convdiff_csr(cd)
    scale = 2.0 ** 130
    op = kr.Operator(cd.n, rp, ci, v * scale)
    B = gaussian_block(cd.n, 4, seed=9)
    A = oracle.csr_matrix_from_arrays(cd.n, rp, ci, v)
    X_lu = splu(A.tocsc()).solve(B) / scale
    X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10, maxit=3000,
                          precision=kr.FP32_REFINE)
    assert info.status == "OK", info
    assert info.fp64_iters > 0 and info.outer_iters == 2, info
    X = host(X)
    assert np.linalg.norm(B - scale * (A @ X)) / np.linalg.norm(B) <= 1.01e-10
    assert np.linalg.norm(X - X_lu) / np.linalg.norm(X_lu) < 1e-8
    op.close()


@pytest.mark.parametrize("s", [4, 8, 16, 32])
@pytest.mark.parametrize("kind", ["gram", "trace"])
@pytest.mark.parametrize("adj", [False, True])
def test_c64_tile_product_full_size(kr, s, kind, adj):
    """128^3 convection-diffusion (the benchmark's matrix, 14.6M entries): the tile kernel's
    product with a fused Gram or trace against FP64 on the host from the complex64 inputs, on
    the rows of a seeded sample and in full for the reduction; products bitwise equal to the
    column-pair kernel's."""
    cd = ConvDiff((128, 128, 128), (0.8, 0.8, 0.8), 0.05j)
    rp, ci, v = convdiff_csr(cd)
    n = cd.n
    op = kr.Operator(n, rp, ci, v)
    g = torch.Generator(device="cuda").manual_seed(s)
    Vd = torch.randn(n, s, dtype=torch.complex64, device="cuda", generator=g)
    Ud = torch.randn(n, s, dtype=torch.complex64, device="cuda", generator=g)
    Y, out = kr.kr_op_apply_reduce_c64(op, Vd, Ud, kind=kind, adjoint=adj)
    Yp, _ = with_pairs(kr, True, lambda: kr.kr_op_apply_reduce_c64(op, Vd, adjoint=adj))
    assert torch.equal(Y, Yp)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, c64(v))
    M = oracle.adjoint(A) if adj else A
    V, U, Yh = host(Vd), host(Ud), host(Y)
    rows = np.random.default_rng(s).integers(0, n, 3000)
    Ms = M[rows]
    ref = Ms @ V
    scale = abs(Ms) @ np.abs(V)
    assert np.all(np.abs(Yh[rows] - ref) <= 4 * 9 * U32 * scale)
    if kind == "gram":
        want, bound = U.conj().T @ Yh, np.abs(U).T @ np.abs(Yh)
    else:
        want, bound = np.array([np.sum(U.conj() * Yh)]), np.array([np.sum(np.abs(U) * np.abs(Yh))])
    got = host(out).reshape(want.shape)
    assert np.all(np.abs(got - want) <= 1e-4 * bound)
    op.close()


@pytest.mark.parametrize("s", [4, 8, 16, 32])
@pytest.mark.parametrize("kind", ["gram", "trace"])
def test_c64_tile_stencil_reductions(kr, s, kind):
    """The tile kernel on the matrix-free stencil (no staged matrix): the product bitwise equal to
    the CSR storage's, the fused Gram / trace against FP64 on the host from the complex64 inputs."""
    cd = ConvDiff((37, 21, 19), (0.4, -0.3, 0.2), 0.05j)
    rp, ci, v = convdiff_csr(cd)
    centre, minus, plus = cd.coefficients()
    st = kr.Operator.stencil(cd.dims, centre, minus, plus)
    csr = kr.Operator(cd.n, rp, ci, v)
    V = c64(gaussian_block(cd.n, s, seed=s))
    U = c64(gaussian_block(cd.n, s, seed=s + 1))
    Ys, outs = kr.kr_op_apply_reduce_c64(st, dev32(V), dev32(U), kind=kind)
    Yc, outc = kr.kr_op_apply_reduce_c64(csr, dev32(V), dev32(U), kind=kind)
    assert torch.equal(Ys, Yc)
    Yk = host(Ys)
    if kind == "gram":
        want, bound = U.conj().T @ Yk, np.abs(U).T @ np.abs(Yk)
    else:
        want, bound = np.array([np.sum(U.conj() * Yk)]), np.array([np.sum(np.abs(U) * np.abs(Yk))])
    for out in (outs, outc):
        got = host(out).reshape(want.shape)
        assert np.all(np.abs(got - want) <= 1e-4 * bound)
    st.close()
    csr.close()


def test_no_device_wait_ran_out(kr):
    assert kr.kr_take_device_timeouts(reset=False) == 0
