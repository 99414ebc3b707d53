"""Matrix-free stencil operator (GPU): same products as the CSR storage of the same stencil.

The stencil kernel applies the entries in the order of the real-off-diagonal CSR
storage (centre, then the minus neighbours from the slowest axis down, then the
plus neighbours), so with real neighbour coefficients its products, and a whole
solve, are bitwise identical to the CSR path; with complex coefficients it is
compared with the oracle's sparse product.
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
    return m


def pair(kr, dims, pe, shift):
    op = ConvDiff(dims, pe, shift)
    rp, ci, v = convdiff_csr(op)
    centre, minus, plus = op.coefficients()
    st = kr.Operator.stencil(dims, centre, minus, plus)
    csr = kr.Operator(op.n, rp, ci, v)
    return op, st, csr, oracle.csr_matrix_from_arrays(op.n, rp, ci, v)


@pytest.mark.parametrize("dims", [(37,), (19, 23), (9, 7, 13), (64, 64, 64)])
@pytest.mark.parametrize("s", [1, 3, 8])
def test_stencil_equals_csr_bitwise(kr, dims, s):
    op, st, csr, A = pair(kr, dims, tuple([0.4, -0.3, 0.2][: len(dims)]), 0.05j)
    assert st.info()["nnz"] == len(A.data) and st.info()["real_offdiag"]
    V = torch.from_numpy(gaussian_block(op.n, s, seed=s)).cuda()
    for adj in (False, True):
        Ys = kr.kr_op_apply(st, V, adjoint=adj)
        Yc = kr.kr_op_apply(csr, V, adjoint=adj)
        assert torch.equal(Ys, Yc), (dims, s, adj)
    st.close()
    csr.close()


def test_stencil_complex_coefficients(kr):
    dims = (11, 8, 6)
    n = int(np.prod(dims))
    centre, minus, plus = 6 + 0.3j, [-1 + 0.2j, -0.7 - 0.1j, -1.1j], [-0.5j, -1 + 0.05j, -0.9]
    st = kr.Operator.stencil(dims, centre, minus, plus)
    assert not st.info()["real_offdiag"]
    # the same matrix assembled densely on the host
    Ad = np.zeros((n, n), dtype=np.complex128)
    strides = [1, dims[0], dims[0] * dims[1]]
    for i in range(n):
        x = [i % dims[0], (i // dims[0]) % dims[1], i // (dims[0] * dims[1])]
        Ad[i, i] = centre
        for a in range(3):
            if x[a] > 0:
                Ad[i, i - strides[a]] = minus[a]
            if x[a] < dims[a] - 1:
                Ad[i, i + strides[a]] = plus[a]
    V = gaussian_block(n, 4, seed=1)
    for adj, M in ((False, Ad), (True, Ad.conj().T)):
        Y = kr.kr_op_apply(st, torch.from_numpy(V).cuda(), adjoint=adj).cpu().numpy()
        ref = M @ V
        assert np.max(np.abs(Y - ref)) <= 1e-14 * np.max(np.abs(M) @ np.abs(V))
    st.close()


@pytest.mark.parametrize("method", ["egl_bicg", "bl_bicg_rq", "gl_qmr"])
def test_stencil_solve_equals_csr_solve(kr, method):
    op, st, csr, A = pair(kr, (16, 16, 16), (0.8, 0.8, 0.8), 0.05j)
    B = torch.from_numpy(gaussian_block(op.n, 4, seed=2)).cuda()
    # matrix-free operators run the algorithms' own order (no fused-product schedule): the same
    # order as the CSR storage's solve with the fused schedule switched off
    Xs, i1 = kr.kr_solve(st, method, B, tol=1e-8, maxit=400)
    kr.kr_set_fused_products(False)
    try:
        Xc, i2 = kr.kr_solve(csr, method, B, tol=1e-8, maxit=400)
    finally:
        kr.kr_set_fused_products(True)
    assert i1.iters == i2.iters and i1.history == i2.history
    assert torch.equal(Xs, Xc)
    ref = oracle.solve(method, A, B.cpu().numpy(), tol=1e-8, maxit=400)
    assert np.allclose(i1.history[:20], ref.history[:20], rtol=1e-10, atol=0)
    st.close()
    csr.close()


def test_stencil_mixed_precision_and_unsupported(kr):
    op, st, csr, A = pair(kr, (12, 12, 12), (0.5, 0.5, 0.5), 0.3j)
    B = gaussian_block(op.n, 8, seed=3)
    X, info = kr.kr_solve(st, "egl_bicg", torch.from_numpy(B).cuda(), tol=1e-10, maxit=1000,
                          precision=kr.FP32_REFINE)
    assert info.status == "OK" and info.outer_iters >= 2
    assert np.linalg.norm(B - A @ X.cpu().numpy()) / np.linalg.norm(B) <= 1e-10
    with pytest.raises(kr.KrylovError, match="UNSUPPORTED"):
        kr.kr_grad_values(st, torch.from_numpy(B).cuda(), torch.from_numpy(B).cuda())
    st.close()
    csr.close()
