"""Mixed-precision solves (GPU) with each complex64 product kernel.

The complex64 inner solves of the iterative refinement (Sec. 1 of the paper: the block
product reads the matrix once for all s columns) run on the row-tile kernel by default;
with it switched off they run on the column-pair kernel.  Both products are bitwise
equal and their reductions agree to FP32 rounding, so both refinements must reach the
requested FP64 residual, checked against the oracle's own residual of the returned X.
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
    yield m
    m.kr_set_tile_kernels(True)


@pytest.mark.parametrize("tile", [True, False])
@pytest.mark.parametrize("s", [4, 8, 16])
def test_mixed_refinement_each_product_kernel(kr, tile, s):
    op_ = ConvDiff((24, 24, 24), (0.8, 0.8, 0.8), 0.05j)
    rp, ci, v = convdiff_csr(op_)
    A = oracle.csr_matrix_from_arrays(op_.n, rp, ci, v)
    B = gaussian_block(op_.n, s, seed=s)
    op = kr.Operator(op_.n, rp, ci, v)
    kr.kr_set_tile_kernels(tile)
    try:
        X, info = kr.kr_solve(op, "egl_bicg", torch.from_numpy(B).cuda(), tol=1e-10, maxit=2000,
                              precision=kr.FP32_REFINE)
    finally:
        kr.kr_set_tile_kernels(True)
        op.close()
    Xh = X.cpu().numpy()
    res = np.linalg.norm(B - oracle.spmm(A, Xh)) / np.linalg.norm(B)
    assert info.status == "OK", info
    assert res <= 2e-10, res
