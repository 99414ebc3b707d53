"""Method-level parity of the CUDA solvers against the FP64 oracle (GPU).

For every method (Algorithms 1-5 and the readings of the BiCGStab / QMR
variants, Secs. 2 and 4): per-iteration relative residual norms over the first
20 iterations, the iteration count to convergence, and X after the oracle's
iteration count k*.  Also: dense LU on the 32 x 32 convection-diffusion problem,
edge cases (s = 1, non-power-of-two s, ragged n, zero right-hand side), failure
statuses, the host-buffer path, the adjoint solve, the gradient, and mixed
precision.

The bar.  The plain bar is 1e-10 relative per iteration and 1e-8 relative on X.
On a well-conditioned input (a complex random matrix with a strong diagonal,
test_plain_bar_well_conditioned) every method is held to the plain bar with no
allowance at all.  The block methods' s x s matrices become ill-conditioned on the
convection-diffusion problems (the inexact deflation of Sec. 4), and there two
correct FP64 programs differ by more than 1e-10: the oracle's own history moves
that far when B is perturbed by one ulp.  On those inputs the bar at iteration k is
max(1e-10 rho_k, 10 sens_k), sens_k being that one-ulp movement, with a hard cap:
an iteration where 10 sens_k exceeds 1e-8 rho_k is never compared (no FP64
program can be), the compared window ends before it and must keep at least
MIN_WINDOW iterations, or the test fails.  Each comparison appends one line to the
JSON-lines file named by the environment variable KR_PARITY_TABLE (when set):
method, test, window, worst |delta_k| / rho_k, worst 10 sens_k / rho_k, which bar
bound, and the X error with its bar.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import ConvDiff, convdiff_csr, gaussian_block, random_csr  # noqa: E402

pytestmark = pytest.mark.gpu

METHODS = ["bl_bicg", "bl_bicg_rq", "gl_bicg", "egl_bicg", "li_bicg", "bl_bicgstab", "bl_bicgstab_rq",
           "gl_bicgstab", "li_bicgstab", "gl_qmr", "egl_qmr", "bl_qmr", "li_qmr"]
HIST_RTOL = 1e-10   # per-iteration residual norms, first 20 iterations
X_RTOL = 1e-8       # iterate after k iterations
SENS_FACTOR = 10.0  # allowed multiple of the oracle's own rounding sensitivity
SENS_CAP = 1e-8     # the widened per-iteration bar never exceeds 1e-8 rho_k
X_SENS_CAP = 1e-6   # nor the widened X bar 1e-6
MIN_WINDOW = 10     # compared iterations (0 .. MIN_WINDOW - 1) that must remain under the cap


def record(**row):
    """Append one row of the per-method parity table (KR_PARITY_TABLE, JSON lines)."""
    path = os.environ.get("KR_PARITY_TABLE")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(row) + "\n")


@pytest.fixture(scope="module")
def kr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_04395_gb300 import build
    build.build()
    import paper_1504_04395_gb300 as m
    m.load_library()
    return m


def conv(N, d=2, pe=0.5, shift=0.1j):
    op = ConvDiff(tuple([N] * d), tuple([pe] * d), shift)
    rp, ci, v = convdiff_csr(op)
    return op.n, rp, ci, v


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def run_pair(kr, method, n, rp, ci, v, B, tol=1e-8, maxit=300, shadow=None):
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    ref = oracle.solve(method, A, B, tol=tol, maxit=maxit, shadow=shadow)
    op = kr.Operator(n, rp, ci, v)
    sh = None if shadow is None else torch.from_numpy(np.ascontiguousarray(shadow)).cuda()
    X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=tol, maxit=maxit, shadow=sh, check_every=4)
    return op, ref, X.cpu().numpy(), info


def oracle_sensitivity(method, A, B, maxit, tol=1e-8, shadow=None, k_x=None):
    """How far the oracle moves under one-ulp perturbations of B: (history deltas, X delta at k_x)."""
    rng = np.random.default_rng(2024)
    base = oracle.solve(method, A, B, tol=tol, maxit=maxit, shadow=shadow)
    dh = np.zeros(len(base.history))
    dx = 0.0
    base_x = oracle.solve(method, A, B, tol=0.0, maxit=k_x, shadow=shadow).X if k_x else None
    for _ in range(2):
        Bp = B * (1 + 2.2e-16 * rng.standard_normal(B.shape))
        r = oracle.solve(method, A, Bp, tol=tol, maxit=maxit, shadow=shadow)
        k = min(len(r.history), len(dh))
        dh[:k] = np.maximum(dh[:k], np.abs(np.array(r.history[:k]) - np.array(base.history[:k])))
        if k_x:
            xp = oracle.solve(method, A, Bp, tol=0.0, maxit=k_x, shadow=shadow).X
            dx = max(dx, rel(xp, base_x))
    return dh, dx


def sens_window(ref_hist, sens, upto=20):
    """Iterations 0 .. K-1 at which the oracle's own one-ulp movement stays under the cap."""
    k = min(upto, len(ref_hist))
    if sens is None:
        return k
    b = np.abs(np.array(ref_hist[:k]))
    over = np.nonzero(SENS_FACTOR * np.asarray(sens[:k]) > SENS_CAP * b)[0]
    return int(over[0]) if len(over) else k


def check_history(ref_hist, gpu_hist, upto=20, sens=None, method="", test="", min_window=MIN_WINDOW):
    """Per-iteration parity over the first `upto` iterations; returns the compared window K.

    sens=None: the plain bar |delta_k| <= 1e-10 rho_k.  Otherwise the capped bar
    max(1e-10 rho_k, 10 sens_k) over the window in which 10 sens_k <= 1e-8 rho_k."""
    k = min(upto, len(ref_hist), len(gpu_hist))
    assert k >= 2
    K = min(k, sens_window(ref_hist, sens, upto))
    assert K >= min(min_window, k), (
        "%s: the oracle's own one-ulp sensitivity exceeds %.0e rho_k at iteration %d: this input is too "
        "ill-conditioned for a parity comparison" % (method, SENS_CAP, K))
    a = np.array(gpu_hist[:K])
    b = np.array(ref_hist[:K])
    plain = HIST_RTOL * np.abs(b)
    bar = plain if sens is None else np.maximum(plain, SENS_FACTOR * np.asarray(sens[:K]))
    d = np.abs(a - b)
    widened = SENS_FACTOR * np.asarray(sens[:K]) / np.abs(b) if sens is not None else np.zeros(K)
    record(method=method, test=test, window=int(K), compared_of=int(k), max_rel_delta=float(np.max(d / np.abs(b))),
           max_rel_sens10=float(np.max(widened)), binds="plain" if np.all(bar == plain) else "sensitivity")
    assert np.all(d <= bar), (method, np.max(d / np.abs(b)), np.max(d - bar))
    return K


def check_x(method, test, X_gpu, X_ref, sens_x=None):
    err = rel(X_gpu, X_ref)
    bar = X_RTOL
    if sens_x is not None:
        assert SENS_FACTOR * sens_x <= X_SENS_CAP, (method, sens_x)
        bar = max(X_RTOL, SENS_FACTOR * sens_x)
    record(method=method, test=test + ":X", x_rel_err=float(err), x_bar=float(bar),
           binds="plain" if bar == X_RTOL else "sensitivity")
    assert err <= bar, (method, err, bar)


@pytest.mark.parametrize("method", METHODS)
def test_method_parity_2d(kr, method):
    """2D convection-diffusion 24 x 24 (n = 576), Pe 0.5, shift 0.3i, s = 4."""
    n, rp, ci, v = conv(24, shift=0.3j)
    B = gaussian_block(n, 4, seed=0)
    op, ref, X, info = run_pair(kr, method, n, rp, ci, v, B)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    sens_h, _ = oracle_sensitivity(method, A, B, 300)
    K = check_history(ref.history, info.history, sens=sens_h, method=method, test="conv2d_24")
    if ref.status == oracle.Status.OK:
        assert info.status == "OK"
        assert abs(info.iters - ref.iters) <= 1, (info.iters, ref.iters)
    # X after exactly k iterations: the oracle's count k* (at most 60) when the whole 20-iteration
    # window was compared, otherwise the last compared iteration (beyond it the oracle's own
    # rounding moves the iterate by more than the cap)
    k = min(ref.iters, 60) if K >= min(20, len(ref.history)) else K - 1
    _, sens_x = oracle_sensitivity(method, A, B, 300, k_x=k)
    ref_k = oracle.solve(method, A, B, tol=0.0, maxit=k)
    Xk, ik = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=0.0, maxit=k)
    assert ik.iters == k
    check_x(method, "conv2d_24@%d" % k, Xk.cpu().numpy(), ref_k.X, sens_x)
    op.close()


@pytest.mark.parametrize("method", METHODS)
def test_plain_bar_well_conditioned(kr, method):
    """The plain bar with no sensitivity allowance: per-iteration residual norms to 1e-10 relative
    and X at the oracle's iteration count to 1e-8, on a well-conditioned input: a random matrix
    with complex off-diagonal entries, empty rows and diagonal shift 6 + 2i (n = 777), s = 3,
    tol 1e-10.  The comparison covers the first 20 iterations, or fewer where the oracle's own
    one-ulp movement (times 10) passes 1e-10 rho_k: the recursive residual of any FP64 program
    carries an absolute error of order eps ||R_0||, which at rho_k ~ 1e-6 is already 1e-10
    relative.  That window must keep 12 iterations (BiCGStab variants converge in 16 here).
    Bl-QMR without look-ahead loses bi-orthogonality by about a digit per iteration, so its
    window ends near iteration 7 and it must keep 6."""
    n = 777
    rp, ci, v = random_csr(n, max_row=6, seed=5, diag_shift=6.0 + 2.0j)
    B = gaussian_block(n, 3, seed=1)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    op, ref, X, info = run_pair(kr, method, n, rp, ci, v, B, tol=1e-10, maxit=300)
    sens_h, _ = oracle_sensitivity(method, A, B, 300, tol=1e-10)
    kk = min(20, len(ref.history))
    relsens = SENS_FACTOR * sens_h[:kk] / np.abs(np.array(ref.history[:kk]))
    over = np.nonzero(relsens > HIST_RTOL)[0]
    K = int(over[0]) if len(over) else kk
    assert K >= (6 if method == "bl_qmr" else 12), (method, K)
    check_history(ref.history, info.history, upto=K, sens=None, method=method, test="plain_random777",
                  min_window=K)
    if ref.status == oracle.Status.OK:
        assert info.status == "OK"
        assert abs(info.iters - ref.iters) <= 1, (info.iters, ref.iters)
    k = ref.iters if method != "bl_qmr" else K - 1
    ref_k = oracle.solve(method, A, B, tol=0.0, maxit=k)
    Xk, ik = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=0.0, maxit=k)
    assert ik.iters == k
    check_x(method, "plain_random777@%d" % k, Xk.cpu().numpy(), ref_k.X, None)
    op.close()


@pytest.mark.parametrize("method", [m for m in METHODS if m != "bl_qmr"])
def test_config1_dense_lu(kr, method):
    """32 x 32 convection-diffusion, Pe 0.5, shift 0.1i, s = 4 Gaussian (seed 0), tol 1e-8 vs dense LU."""
    n, rp, ci, v = conv(32, pe=0.5, shift=0.1j)
    B = gaussian_block(n, 4, seed=0)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    X_lu = np.linalg.solve(A.toarray(), B)
    op = kr.Operator(n, rp, ci, v)
    X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-8, maxit=1000)
    assert info.status == "OK", info
    assert info.relres_true < 2e-8
    assert rel(X.cpu().numpy(), X_lu) < 1e-6
    ref = oracle.solve(method, A, B, tol=1e-8, maxit=1000)
    check_history(ref.history, info.history, sens=oracle_sensitivity(method, A, B, 1000)[0], method=method,
                  test="config1_32x32")
    op.close()


@pytest.mark.parametrize("s", [1, 3, 5, 12, 16])
@pytest.mark.parametrize("method", ["egl_bicg", "gl_bicg", "bl_bicg", "bl_bicgstab", "gl_qmr", "bl_bicg_rq"])
def test_s_edge_cases(kr, method, s):
    n, rp, ci, v = conv(13, d=3, pe=0.4, shift=0.5j)  # n = 2197: ragged tail for every G
    B = gaussian_block(n, s, seed=s)
    op, ref, X, info = run_pair(kr, method, n, rp, ci, v, B, maxit=200)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    check_history(ref.history, info.history, sens=oracle_sensitivity(method, A, B, 200)[0], method=method,
                  test="conv3d_13_s%d" % s)
    assert info.status == ref.status.name
    op.close()


@pytest.mark.parametrize("method", ["gl_bicg", "egl_bicg", "bl_bicg", "bl_qmr"])
def test_user_shadow(kr, method):
    n, rp, ci, v = conv(20, shift=0.2j)
    B = gaussian_block(n, 3, seed=2)
    shadow = gaussian_block(n, 3, seed=9)
    if method.startswith("egl"):
        shadow = np.ascontiguousarray(shadow[:, 0])
    op, ref, X, info = run_pair(kr, method, n, rp, ci, v, B, maxit=100, shadow=shadow)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    check_history(ref.history, info.history, sens=oracle_sensitivity(method, A, B, 100, shadow=shadow)[0],
                  method=method, test="user_shadow")
    op.close()


def test_statuses(kr):
    n, rp, ci, v = conv(12, shift=0.3j)
    op = kr.Operator(n, rp, ci, v)
    B = gaussian_block(n, 3, seed=1)
    # duplicate columns: singular s x s matrices in Bl-BiCG (Sec. 2)
    Bd = B.copy()
    Bd[:, 2] = Bd[:, 1]
    _, info = kr.kr_solve(op, "bl_bicg", torch.from_numpy(Bd).cuda(), tol=1e-10, maxit=50)
    assert info.status == "BREAKDOWN"
    Bn = B.copy()
    Bn[5, 0] = np.nan
    _, info = kr.kr_solve(op, "gl_bicg", torch.from_numpy(Bn).cuda(), tol=1e-10, maxit=10)
    assert info.status == "NAN"
    _, info = kr.kr_solve(op, "egl_bicg", torch.from_numpy(B).cuda(), tol=1e-15, maxit=3)
    assert info.status == "MAXIT" and info.iters == 3
    X, info = kr.kr_solve(op, "egl_qmr", torch.zeros((n, 3), dtype=torch.complex128, device="cuda"), tol=1e-10)
    assert info.status == "OK" and info.iters == 0 and float(X.abs().max()) == 0.0
    op.close()


def test_host_buffers_match_device(kr):
    n, rp, ci, v = conv(20, shift=0.2j)
    B = gaussian_block(n, 4, seed=4)
    op = kr.Operator(n, rp, ci, v)
    Xd, i1 = kr.kr_solve(op, "egl_bicg", torch.from_numpy(B).cuda(), tol=1e-9, maxit=200)
    Xh, i2 = kr.kr_solve(op, "egl_bicg", torch.from_numpy(B).pin_memory(), tol=1e-9, maxit=200)
    assert not Xh.is_cuda
    assert i1.iters == i2.iters
    assert torch.equal(Xd.cpu(), Xh)
    op.close()


@pytest.mark.parametrize("method", ["egl_bicg", "gl_bicg", "bl_bicg"])
def test_adjoint_solve(kr, method):
    n, rp, ci, v = conv(16, shift=0.2j)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    G = gaussian_block(n, 3, seed=6)
    op = kr.Operator(n, rp, ci, v)
    L, info = kr.kr_adjoint_solve(op, method, torch.from_numpy(G).cuda(), tol=1e-11, maxit=400)
    assert info.status == "OK"
    L_ref = np.linalg.solve(A.toarray().conj().T, G)
    assert rel(L.cpu().numpy(), L_ref) < 1e-8
    ref = oracle.solve(method, oracle.adjoint(A), G, tol=1e-11, maxit=400)
    check_history(ref.history, info.history, sens=oracle_sensitivity(method, oracle.adjoint(A), G, 400, tol=1e-11)[0],
                  method=method, test="adjoint")
    op.close()


def test_grad_values(kr):
    n = 300
    rp, ci, v = random_csr(n, seed=3)
    Lam = gaussian_block(n, 5, seed=1)
    X = gaussian_block(n, 5, seed=2)
    op = kr.Operator(n, rp, ci, v)
    dv = kr.kr_grad_values(op, torch.from_numpy(Lam).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    ref = -np.sum(Lam[rows] * np.conj(X[ci]), axis=1)
    assert np.max(np.abs(dv - ref)) < 1e-13 * np.max(np.abs(ref))
    op.close()


@pytest.mark.parametrize("method", ["egl_bicg", "gl_bicgstab", "bl_bicgstab"])
def test_mixed_precision_refinement(kr, method):
    """complex64 inner solves (tol 1e-4) inside FP64 defect correction to 1e-10."""
    n, rp, ci, v = conv(10, d=3, pe=0.5, shift=0.3j)
    B = gaussian_block(n, 8, seed=3)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    op = kr.Operator(n, rp, ci, v)
    X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10, maxit=1000,
                          precision=kr.FP32_REFINE, inner_tol=1e-4)
    assert info.status == "OK", info
    assert info.outer_iters >= 2
    Xn = X.cpu().numpy()
    assert np.linalg.norm(B - A @ Xn) / np.linalg.norm(B) <= 1e-10
    X_lu = np.linalg.solve(A.toarray(), B)
    assert rel(Xn, X_lu) < 1e-8
    op.close()


@pytest.mark.parametrize("method", ["egl_bicg", "gl_bicg", "bl_bicg", "bl_bicg_rq", "bl_bicgstab", "gl_qmr"])
def test_orthonormalize_B(kr, method):
    """kr_options.orthonormalize_B (the set-up of Sec. 5: B - A X_0 = Q S, solve A Y = Q, X = X_0 + Y S)
    against the oracle with the same option: the history of the system with Q, X after the
    oracle's iteration count, and the solution against dense LU; from a non-zero X_0."""
    n, rp, ci, v = conv(20, shift=0.3j)
    B = gaussian_block(n, 4, seed=11)
    X0 = 0.1 * gaussian_block(n, 4, seed=12)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    ref = oracle.solve(method, A, B, X0=X0, tol=1e-10, maxit=400, orthonormalize_B=True)
    op = kr.Operator(n, rp, ci, v)
    X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), X=torch.from_numpy(X0.copy()).cuda(), tol=1e-10,
                          maxit=400, orthonormalize_B=True, check_every=4)
    assert info.status == "OK" == ref.status.name, (info, ref.status)
    assert abs(info.iters - ref.iters) <= 1
    # sensitivity of the oracle's own history with the orthonormalised set-up (one-ulp changes of B)
    rng = np.random.default_rng(2024)
    sens = np.zeros(len(ref.history))
    for _ in range(2):
        Bp = B * (1 + 2.2e-16 * rng.standard_normal(B.shape))
        rp_ = oracle.solve(method, A, Bp, X0=X0, tol=1e-10, maxit=400, orthonormalize_B=True)
        k = min(len(rp_.history), len(sens))
        sens[:k] = np.maximum(sens[:k], np.abs(np.array(rp_.history[:k]) - np.array(ref.history[:k])))
    check_history(ref.history, info.history, sens=sens, method=method, test="orthonormalize_B")
    assert info.relres_true <= 2e-10
    Xd = np.linalg.solve(A.toarray(), B)
    assert rel(X.cpu().numpy(), Xd) < 1e-7
    k = ref.iters
    ref_k = oracle.solve(method, A, B, X0=X0, tol=0.0, maxit=k, orthonormalize_B=True)
    Xk, ik = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), X=torch.from_numpy(X0.copy()).cuda(), tol=0.0,
                         maxit=k, orthonormalize_B=True)
    check_x(method, "orthonormalize_B@%d" % k, Xk.cpu().numpy(), ref_k.X, None)
    op.close()


def test_breakdown_iter_and_rank_deficient_rhs(kr):
    n, rp, ci, v = conv(12, shift=0.3j)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    op = kr.Operator(n, rp, ci, v)
    B = gaussian_block(n, 3, seed=1)
    B[:, 2] = B[:, 1]
    ref = oracle.solve("bl_bicg", A, B, tol=1e-10, maxit=50)
    _, info = kr.kr_solve(op, "bl_bicg", torch.from_numpy(B).cuda(), tol=1e-10, maxit=50)
    assert info.status == "BREAKDOWN" == ref.status.name
    assert info.breakdown_iter == ref.breakdown_iter == info.iters + 1
    _, info = kr.kr_solve(op, "gl_bicg", torch.from_numpy(B).cuda(), tol=1e-10, maxit=50, orthonormalize_B=True)
    assert info.status == "BREAKDOWN" and info.breakdown_iter == 1 and info.iters == 0
    _, info = kr.kr_solve(op, "gl_bicg", torch.from_numpy(gaussian_block(n, 3, seed=2)).cuda(), tol=1e-10, maxit=300)
    assert info.status == "OK" and info.breakdown_iter == 0
    op.close()


def test_create_csr_from_device_arrays(kr):
    """kr_op_create_csr_async with device arrays on a side stream builds the operator that
    kr_op_create_csr builds from the same arrays on the host: bitwise equal products."""
    n = 3001
    rp, ci, v = random_csr(n, max_row=7, seed=9, diag_shift=4.0 + 1.0j)
    ref = kr.Operator(n, rp, ci, v)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        rpt = torch.from_numpy(np.asarray(rp, dtype=np.int64)).cuda()
        cit = torch.from_numpy(np.asarray(ci, dtype=np.int32)).cuda()
        vt = torch.from_numpy(np.asarray(v, dtype=np.complex128)).cuda()
        op = kr.Operator.from_tensors(rpt, cit, vt, stream=side)
    side.synchronize()
    assert op.info() == ref.info()
    V = torch.from_numpy(gaussian_block(n, 5, seed=3)).cuda()
    for adj in (False, True):
        assert torch.equal(kr.kr_op_apply(op, V, adjoint=adj), kr.kr_op_apply(ref, V, adjoint=adj))
    host = kr.Operator.from_tensors(torch.from_numpy(np.asarray(rp, dtype=np.int64)),
                                    torch.from_numpy(np.asarray(ci, dtype=np.int32)),
                                    torch.from_numpy(np.asarray(v, dtype=np.complex128)))
    assert torch.equal(kr.kr_op_apply(host, V), kr.kr_op_apply(ref, V))
    bad = cit.clone()
    bad[7] = n  # out of range: rejected on the host after the copy, before any GPU work on it
    with pytest.raises(kr.KrylovError):
        kr.Operator.from_tensors(rpt, bad, vt)
    for o in (op, ref, host):
        o.close()


@pytest.mark.parametrize("method", ["gl_bicg", "egl_bicg"])
def test_fused_schedule_against_oracle_and_literal(kr, method):
    """Gl-/eGl-BiCG with alpha from the adjoint product and the X / R update fused with A P
    (kr_set_fused_products, the default) against the oracle's Algorithms 2 and 4 (the plain bar),
    against the literal schedule of the same library, and the bytes each moves per iteration
    (launch profile: 2M + 8 Bv instead of 2M + 11 Bv for eGl-BiCG)."""
    n, rp, ci, v = conv(24, shift=0.3j)
    B = gaussian_block(n, 4, seed=0)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    ref = oracle.solve(method, A, B, tol=1e-8, maxit=300)
    op = kr.Operator(n, rp, ci, v)
    runs = {}
    for fused in (True, False):
        kr.kr_set_fused_products(fused)
        try:
            runs[fused] = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-8, maxit=300)
        finally:
            kr.kr_set_fused_products(True)
    (Xf, inf_f), (Xl, inf_l) = runs[True], runs[False]
    check_history(ref.history, inf_f.history, sens=None, method=method, test="fused_schedule")
    assert inf_f.status == "OK" and inf_f.iters == ref.iters == inf_l.iters
    assert rel(Xf.cpu().numpy(), Xl.cpu().numpy()) < 1e-9
    assert rel(Xf.cpu().numpy(), ref.X) < 1e-9
    # bytes per iteration, from the launch profile of 10-iteration solves
    per_iter = {}
    for fused in (True, False):
        kr.kr_set_fused_products(fused)
        try:
            for k in (5, 15):
                kr.kr_profile_read(reset=True)
                kr.kr_profile_enable(True, time_kernels=False)
                kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=0.0, maxit=k, graphs="off")
                prof = kr.kr_profile_read(reset=True)
                kr.kr_profile_enable(False)
                per_iter[(fused, k)] = sum(c["bytes"] for c in prof.values())
        finally:
            kr.kr_set_fused_products(True)
    fused_b = (per_iter[(True, 15)] - per_iter[(True, 5)]) / 10
    literal_b = (per_iter[(False, 15)] - per_iter[(False, 5)]) / 10
    s = 4
    Bv = 16.0 * n * s
    saved = (literal_b - fused_b) / Bv
    # eGl-BiCG: three blocks fewer, two n-vectors (1/s of a block each) more; Gl-BiCG: two blocks fewer
    assert saved == pytest.approx(3.0 - 2.0 / s if method == "egl_bicg" else 2.0, abs=0.02), saved
    op.close()


@pytest.mark.parametrize("kind", ["stencil", "lattice", "ilu0", "mixed"])
def test_fused_schedule_other_operators(kr, kind):
    """eGl-BiCG with fused products on (the default) on the other operators: the matrix-free stencil
    (which runs the algorithms' own order), the matrix-free lattice and the ILU(0)-preconditioned
    CSR operator (fused schedule, product stored first, then combined), and in mixed precision
    (complex64 inner solves): against the oracle or dense LU."""
    method = "egl_bicg"
    if kind == "lattice":
        from workloads import Lattice4D, lattice_csr
        from workloads.lattice import GAMMA, LATTICE_MASS, haar_links
        lat = Lattice4D((4, 4, 4, 4), LATTICE_MASS, seed=0)
        links = haar_links(lat.dims, lat.seed)
        rp, ci, v = lattice_csr(lat, links)
        n = lat.n
        op = kr.Operator.lattice4d(lat.dims, 4.0 + LATTICE_MASS, -0.5, GAMMA, links)
    else:
        cd = ConvDiff((10, 10, 10), (0.4, 0.4, 0.4), 0.3j)
        rp, ci, v = convdiff_csr(cd)
        n = cd.n
        if kind == "stencil":
            centre, minus, plus = cd.coefficients()
            op = kr.Operator.stencil(cd.dims, centre, minus, plus)
        else:
            op = kr.Operator(n, rp, ci, v)
            if kind == "ilu0":
                op.set_preconditioner("ilu0")
    B = gaussian_block(n, 4, seed=3)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    if kind == "mixed":
        X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10, maxit=1000,
                              precision=kr.FP32_REFINE)
        assert info.status == "OK" and info.fp64_iters == 0, info
        assert rel(X.cpu().numpy(), np.linalg.solve(A.toarray(), B)) < 1e-8
    elif kind == "ilu0":
        X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10, maxit=500)
        assert info.status == "OK"
        assert rel(X.cpu().numpy(), np.linalg.solve(A.toarray(), B)) < 1e-8
    else:
        ref = oracle.solve(method, A, B, tol=1e-10, maxit=1000)
        X, info = kr.kr_solve(op, method, torch.from_numpy(B).cuda(), tol=1e-10, maxit=1000)
        assert info.status == "OK" and abs(info.iters - ref.iters) <= 1
        check_history(ref.history, info.history, sens=None, method=method, test="fused_" + kind)
    op.close()
