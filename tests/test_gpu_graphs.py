"""CUDA-graph replay of the solver iterations (GPU).

With `graphs="on"` iteration 0 runs eagerly, iterations 1 and 2 are captured on a private
stream and the graph is replayed until the device state reports completion.  The same
kernels run in the same order with the same arguments, so iterates, residual histories,
iteration counts and statuses are bitwise those of the eager launches.
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


def problem(kr, N=24, s=4):
    op = ConvDiff((N, N), (0.5, 0.5), 0.3j)
    rp, ci, v = convdiff_csr(op)
    return kr.Operator(op.n, rp, ci, v), gaussian_block(op.n, s, seed=0), (op.n, rp, ci, v)


METHODS = ["egl_bicg", "gl_bicg", "li_bicg", "bl_bicg", "bl_bicg_rq", "bl_bicgstab", "bl_bicgstab_rq",
           "gl_bicgstab", "li_bicgstab", "gl_qmr", "egl_qmr", "bl_qmr", "li_qmr"]


@pytest.mark.parametrize("method", METHODS)
def test_graph_replay_is_bitwise_eager(kr, method):
    op, B, _ = problem(kr)
    Bd = torch.from_numpy(B).cuda()
    Xe, ie = kr.kr_solve(op, method, Bd, tol=1e-8, maxit=300, graphs="off")
    Xg, ig = kr.kr_solve(op, method, Bd, tol=1e-8, maxit=300, graphs="on")
    assert (ie.status, ie.iters) == (ig.status, ig.iters)
    assert torch.equal(Xe, Xg)
    assert ie.history == ig.history
    op.close()


@pytest.mark.parametrize("maxit", [1, 2, 3, 4, 5, 8, 9])
def test_graph_replay_exact_iteration_limits(kr, maxit):
    """The iteration count is exact for any maxit (replays past the limit are no-ops)."""
    op, B, _ = problem(kr)
    Bd = torch.from_numpy(B).cuda()
    for check_every in (1, 8):
        Xe, ie = kr.kr_solve(op, "bl_bicg", Bd, tol=0.0, maxit=maxit, graphs="off", check_every=check_every)
        Xg, ig = kr.kr_solve(op, "bl_bicg", Bd, tol=0.0, maxit=maxit, graphs="on", check_every=check_every)
        assert ie.iters == ig.iters == maxit
        assert torch.equal(Xe, Xg)
    op.close()


def test_graph_replay_on_a_side_stream_and_with_mixed_precision(kr):
    op, B, (n, rp, ci, v) = problem(kr)
    Bd = torch.from_numpy(B).cuda()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        Xs, is_ = kr.kr_solve(op, "egl_bicg", Bd, tol=1e-10, maxit=500, graphs="on", stream=side)
    side.synchronize()
    Xe, ie = kr.kr_solve(op, "egl_bicg", Bd, tol=1e-10, maxit=500, graphs="off")
    assert torch.equal(Xs, Xe) and is_.iters == ie.iters
    Xm, im = kr.kr_solve(op, "egl_bicg", Bd, tol=1e-10, maxit=1000, precision=kr.FP32_REFINE, graphs="on")
    Xo, io = kr.kr_solve(op, "egl_bicg", Bd, tol=1e-10, maxit=1000, precision=kr.FP32_REFINE, graphs="off")
    assert torch.equal(Xm, Xo) and im.iters == io.iters and im.status == io.status == "OK"
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    assert np.linalg.norm(B - A @ Xm.cpu().numpy()) / np.linalg.norm(B) <= 1.01e-10
    op.close()


def test_graph_replay_off_while_profiling(kr):
    """The launch profile counts host-side launches, so a profiled solve runs eagerly."""
    op, B, _ = problem(kr)
    Bd = torch.from_numpy(B).cuda()
    kr.kr_profile_read(reset=True)
    kr.kr_profile_enable(True)
    try:
        _, info = kr.kr_solve(op, "gl_bicg", Bd, tol=0.0, maxit=10, graphs="on")
        prof = kr.kr_profile_read(reset=True)
    finally:
        kr.kr_profile_enable(False)
    assert info.iters == 10
    # every iteration's launches were counted: one product launch and two row-local launches
    # per iteration at least (the fused schedule forms A P inside a row-local launch)
    assert prof["spmm"]["launches"] >= 10 and prof["lincomb"]["launches"] >= 2 * 10
    op.close()


def test_graph_replay_is_faster_on_a_small_problem(kr):
    """Config 1 size (32 x 32, s = 4): the iterations are launch-bound without graphs."""
    import time
    op, B, _ = problem(kr, N=32)
    Bd = torch.from_numpy(B).cuda()
    t = {}
    for mode in ("off", "on"):
        kr.kr_solve(op, "bl_bicg", Bd, tol=0.0, maxit=50, graphs=mode)
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(3):
            t0 = time.perf_counter()
            kr.kr_solve(op, "bl_bicg", Bd, tol=0.0, maxit=200, graphs=mode)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        t[mode] = best
    assert t["on"] < t["off"], t
    op.close()
