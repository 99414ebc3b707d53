"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics (CPU only).

Each test names the passage of the paper (section, algorithm, equation or
table) it follows.  None of them compares the oracle with a retyped copy of
itself: the references are dense LU solutions, the classical single-RHS
methods, the Kronecker form of the global methods, brute-force Petrov-Galerkin
and quasi-minimal-residual solutions built from dense bases, exact identities
between methods, and the numbers printed in Table 1.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import Status
from oracle.ops import thin_qr
from workloads import ConvDiff, convdiff_csr, gaussian_block, grid_nnz, Lattice4D, lattice_csr

HERE = os.path.dirname(os.path.abspath(__file__))

BICG_LIKE = ["bl_bicg", "bl_bicg_rq", "gl_bicg", "egl_bicg", "li_bicg"]
STAB_LIKE = ["bl_bicgstab", "bl_bicgstab_rq", "gl_bicgstab", "li_bicgstab"]
QMR_LIKE = ["gl_qmr", "egl_qmr", "bl_qmr", "li_qmr"]
ALL = BICG_LIKE + STAB_LIKE + QMR_LIKE


def problem(N=10, d=2, pe=0.3, shift=0.5j, s=3, seed=1):
    op = ConvDiff(tuple([N] * d), tuple([pe] * d), shift)
    rp, ci, v = convdiff_csr(op)
    A = oracle.csr_matrix_from_arrays(op.n, rp, ci, v)
    B = gaussian_block(op.n, s, seed)
    return A, B


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def vec(X):
    """vec of Sec. 2: (X)_ij = x_{(j-1)n+i}, i.e. columns stacked."""
    return np.asarray(X).reshape(-1, order="F")


def kron_I(A, s):
    import scipy.sparse as sp
    return sp.kron(sp.identity(s, dtype=np.complex128, format="csr"), A, format="csr")


# ------------------------------------------------------------------------------------------
# Table 1 and the example descriptions of Sec. 5
# ------------------------------------------------------------------------------------------

def test_table1_rho_and_sizes():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_rho.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            ex, grid, s, rho = line.split()
            rows.append((ex, tuple(int(g) for g in grid.split("x")), int(s), float(rho)))
    assert len(rows) == 4
    for ex, grid, s, rho_printed in rows:
        if len(grid) == 4:
            lat = Lattice4D(grid, mass=0.1, seed=0)
            rp, ci, v = lattice_csr(lat)
            n, nnz = lat.n, len(v)
            assert n == 49152  # Example 4: 12 * 8^4
            assert nnz == 49 * n  # Example 4: 49 non-zeros per row
            assert np.all(np.diff(rp) == 49)
        else:
            op = ConvDiff(grid, tuple([0.1] * len(grid)), 0.0)
            rp, ci, v = convdiff_csr(op)
            n, nnz = op.n, len(v)
            assert nnz == grid_nnz(grid)
            if ex in ("ex2", "ex3"):
                assert n == 125000
                assert np.max(np.diff(rp)) == 7
        rho = s * n / nnz  # Eq. (rho)
        assert round(rho, 2) == pytest.approx(rho_printed, abs=0.006), (ex, rho)


# ------------------------------------------------------------------------------------------
# the textbook single-RHS methods are themselves pinned
# ------------------------------------------------------------------------------------------

def test_textbook_bicg_pins():
    A, B = problem(N=5, s=1, shift=0.3j)
    Ad = A.toarray()
    n = Ad.shape[0]
    out = oracle.bicg_textbook(Ad, B[:, 0], iters=n)
    xs, rs, rhs = out["x"], out["r"], out["rh"]
    # bi-orthogonality of residuals: rh_j^H r_k = 0 for j != k (early iterations)
    for j in range(6):
        for k in range(6):
            if j != k:
                assert abs(np.vdot(rhs[j], rs[k])) <= 1e-10 * np.linalg.norm(rhs[j]) * np.linalg.norm(rs[k])
    # recursive residual = true residual
    for k in range(8):
        assert rel(rs[k], B[:, 0] - Ad @ xs[k]) < 1e-10
    # finite termination (n steps) in exact arithmetic: the solution up to rounding amplification
    x_lu = np.linalg.solve(Ad, B[:, 0])
    assert rel(xs[n], x_lu) < 1e-6


def test_textbook_bicgstab_pins():
    A, B = problem(N=8, s=1, shift=0.5j)
    Ad = A.toarray()
    out = oracle.bicgstab_textbook(Ad, B[:, 0], iters=60)
    x_lu = np.linalg.solve(Ad, B[:, 0])
    assert rel(out["x"][-1], x_lu) < 1e-10
    for k in range(10):
        assert rel(out["r"][k], B[:, 0] - Ad @ out["x"][k]) < 1e-10


# ------------------------------------------------------------------------------------------
# every method converges to the dense LU solution (Sec. 1: A X = B)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("method", ALL)
def test_dense_lu_tiny(method):
    A, B = problem(N=6, s=3, shift=0.5j)
    X_lu = np.linalg.solve(A.toarray(), B)
    r = oracle.solve(method, A, B, tol=1e-12, maxit=400)
    assert r.status == Status.OK, (method, r.status, r.iters)
    assert r.relres_true < 1e-11
    assert rel(r.X, X_lu) < 1e-9


@pytest.mark.parametrize("method", [m for m in ALL if m != "bl_qmr"])
def test_dense_lu_32x32(method):
    """2D convection-diffusion 32 x 32, Pe 0.5, shift 0.1i, s = 4 (stand-in for Example 1)."""
    A, B = problem(N=32, pe=0.5, shift=0.1j, s=4, seed=0)
    X_lu = np.linalg.solve(A.toarray(), B)
    r = oracle.solve(method, A, B, tol=1e-8, maxit=1000)
    assert r.status == Status.OK
    assert r.relres_true < 2e-8
    # ||X - X_LU|| / ||X_LU|| <= kappa * tol with kappa(A) ~ 80 for this operator
    assert rel(r.X, X_lu) < 1e-6


# ------------------------------------------------------------------------------------------
# Sec. 2: all simultaneous methods reduce to the single-RHS method for s = 1
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("method", BICG_LIKE)
def test_s1_reduces_to_bicg(method):
    A, B = problem(N=8, s=1, shift=0.4j)
    ref = oracle.bicg_textbook(A, B[:, 0], iters=10)
    for k in (1, 2, 5, 10):
        r = oracle.solve(method, A, B, tol=0.0, maxit=k)
        assert r.iters == k
        assert rel(r.X[:, 0], ref["x"][k]) < 1e-10, (method, k)


@pytest.mark.parametrize("method", STAB_LIKE)
def test_s1_reduces_to_bicgstab(method):
    A, B = problem(N=8, s=1, shift=0.4j)
    ref = oracle.bicgstab_textbook(A, B[:, 0], iters=10)
    for k in (1, 2, 5, 10):
        r = oracle.solve(method, A, B, tol=0.0, maxit=k)
        assert rel(r.X[:, 0], ref["x"][k]) < 1e-10, (method, k)


@pytest.mark.parametrize("method", ["egl_qmr", "bl_qmr"])
def test_s1_qmr_variants_agree(method):
    A, B = problem(N=8, s=1, shift=0.4j)
    for k in (1, 3, 8):
        a = oracle.solve(method, A, B, tol=0.0, maxit=k)
        b = oracle.solve("gl_qmr", A, B, tol=0.0, maxit=k)
        assert rel(a.X, b.X) < 1e-10


# ------------------------------------------------------------------------------------------
# Sec. 2, Eq. (global): a global method is the single-RHS method for (I (x) A) vec(X) = vec(B)
# ------------------------------------------------------------------------------------------

def test_global_bicg_is_kron_bicg():
    A, B = problem(N=7, s=3, shift=0.3j)
    K = kron_I(A, 3)
    ref = oracle.bicg_textbook(K, vec(B), iters=12)
    for k in (1, 4, 12):
        r = oracle.solve("gl_bicg", A, B, tol=0.0, maxit=k)
        assert rel(vec(r.X), ref["x"][k]) < 1e-10


def test_global_bicgstab_is_kron_bicgstab():
    A, B = problem(N=7, s=3, shift=0.3j)
    K = kron_I(A, 3)
    ref = oracle.bicgstab_textbook(K, vec(B), iters=12)
    for k in (1, 4, 12):
        r = oracle.solve("gl_bicgstab", A, B, tol=0.0, maxit=k)
        assert rel(vec(r.X), ref["x"][k]) < 1e-10


def test_global_qmr_is_kron_qmr():
    A, B = problem(N=7, s=3, shift=0.3j)
    K = kron_I(A, 3)
    for k in (1, 4, 12):
        r = oracle.solve("gl_qmr", A, B, tol=0.0, maxit=k)
        ref = oracle.solve("gl_qmr", K, vec(B)[:, None], tol=0.0, maxit=k)
        assert rel(vec(r.X), ref.X[:, 0]) < 1e-10


# ------------------------------------------------------------------------------------------
# Sec. 4: identical-column shadows are preserved; eGl-* equals Gl-* with R^_0 = r^_0 1^T
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("pair", [("egl_bicg", "gl_bicg"), ("egl_qmr", "gl_qmr")])
def test_economic_equals_global_with_identical_columns(pair):
    A, B = problem(N=9, s=4, shift=0.3j)
    R0 = B.copy()
    rh = R0.mean(axis=1)  # Sec. 5: arithmetic mean of the initial residuals
    Rh = np.repeat(rh[:, None], 4, axis=1)
    for k in (1, 5, 15):
        e = oracle.solve(pair[0], A, B, tol=0.0, maxit=k)
        g = oracle.solve(pair[1], A, B, tol=0.0, maxit=k, shadow=Rh)
        assert rel(e.X, g.X) < 1e-10
        assert np.allclose(e.history, g.history, rtol=1e-9, atol=0)


# ------------------------------------------------------------------------------------------
# Sec. 2: Petrov-Galerkin characterisation of Bl-BiCG (and of Gl-BiCG on the Kronecker system)
# ------------------------------------------------------------------------------------------

def _pg_iterate(Ad, R0, Rh0, k):
    """X_k - X_0 in K_k(A, R0) with R_k orthogonal to K_k(A^H, Rh0), from dense orthonormal bases."""
    AH = Ad.conj().T
    Ks, Kh = [R0], [Rh0]
    for _ in range(k - 1):
        Ks.append(Ad @ Ks[-1])
        Kh.append(AH @ Kh[-1])
    Kb, _ = np.linalg.qr(np.hstack(Ks))
    Kbh, _ = np.linalg.qr(np.hstack(Kh))
    Z = np.linalg.solve(Kbh.conj().T @ Ad @ Kb, Kbh.conj().T @ R0)
    return Kb @ Z


@pytest.mark.parametrize("method", ["bl_bicg", "bl_bicg_rq"])
def test_block_bicg_petrov_galerkin(method):
    A, B = problem(N=6, s=3, shift=0.3j)
    Ad = A.toarray()
    for k in (1, 2, 3):
        r = oracle.solve(method, A, B, tol=0.0, maxit=k)
        X_pg = _pg_iterate(Ad, B, B, k)
        assert rel(r.X, X_pg) < 1e-9, (method, k)
        # the residual is orthogonal to the shadow block Krylov space
        Rk = B - Ad @ r.X
        Kh = np.hstack([np.linalg.matrix_power(Ad.conj().T, j) @ B for j in range(k)])
        assert np.linalg.norm(Kh.conj().T @ Rk) < 1e-9 * np.linalg.norm(Kh) * np.linalg.norm(Rk)


@pytest.mark.parametrize("method", ["bl_bicg", "bl_bicg_rq"])
def test_block_bicg_petrov_galerkin_complex_offdiagonals(method):
    """The same characterisation on a matrix with complex off-diagonal entries.  For the
    convection-diffusion matrices (real off-diagonals, complex shift on the diagonal) the
    Krylov spaces of A^T and A^H coincide (shift invariance), so only a matrix like this one
    fixes that the shadow recurrence multiplies by A^H."""
    from workloads.random_csr import random_csr
    n, s = 40, 3
    rp, ci, v = random_csr(n, max_row=5, seed=3, empty_frac=0.0)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    B = gaussian_block(n, s, 5)
    Ad = A.toarray()
    for k in (1, 2, 3):
        r = oracle.solve(method, A, B, tol=0.0, maxit=k)
        assert rel(r.X, _pg_iterate(Ad, B, B, k)) < 1e-9, (method, k)


@pytest.mark.parametrize("method", ["bl_bicg", "bl_bicg_rq", "gl_bicg", "li_bicg"])
def test_bicg_biorthogonality(method):
    """Bi-orthogonality of the BiCG residuals (Sec. 2): Rh_j^H R_k = 0 for j != k (block),
    tr(Rh_j^H R_k) = 0 (global), rh_{j,i}^H r_{k,i} = 0 per column (loop interchange).
    BiCG treats its two sequences symmetrically, so the shadow residuals Rh_j are the
    residuals Rh_0 - A^H Xh_j of the same method run on A^H Xh = Rh_0 with shadow R_0."""
    A, B = problem(N=8, s=3, shift=0.3j)
    Rh0 = gaussian_block(B.shape[0], 3, 21)
    AH = oracle.adjoint(A)
    K = 6
    R = [B - A @ oracle.solve(method, A, B, tol=0.0, maxit=k, shadow=Rh0).X for k in range(K)]
    Rh = [Rh0 - AH @ oracle.solve(method, AH, Rh0, tol=0.0, maxit=k, shadow=B).X for k in range(K)]

    def coupling(U, V):
        if method == "gl_bicg":
            return abs(np.vdot(U, V)) / (np.linalg.norm(U) * np.linalg.norm(V))
        if method == "li_bicg":
            return max(abs(np.vdot(U[:, i], V[:, i])) / (np.linalg.norm(U[:, i]) * np.linalg.norm(V[:, i]))
                       for i in range(U.shape[1]))
        return np.linalg.norm(U.conj().T @ V) / (np.linalg.norm(U) * np.linalg.norm(V))

    for j in range(K):
        for k in range(K):
            if j != k:
                assert coupling(Rh[j], R[k]) < 1e-10, (j, k)
    assert coupling(Rh[2], R[2]) > 1e-3  # the pairing itself is not degenerate


def test_global_bicg_petrov_galerkin():
    A, B = problem(N=6, s=3, shift=0.3j)
    K = kron_I(A, 3).toarray()
    for k in (1, 2, 3):
        r = oracle.solve("gl_bicg", A, B, tol=0.0, maxit=k)
        x_pg = _pg_iterate(K, vec(B)[:, None], vec(B)[:, None], k)[:, 0]
        assert rel(vec(r.X), x_pg) < 1e-9


def test_li_bicgstab_is_columnwise_bicgstab():
    """Li-BiCGStab: column i is BiCGStab for A x_i = b_i (loop interchange, Sec. 2)."""
    A, B = problem(N=7, s=3, shift=0.3j)
    r = oracle.solve("li_bicgstab", A, B, tol=0.0, maxit=9)
    for i in range(3):
        ref = oracle.bicgstab_textbook(A, B[:, i], iters=9)
        assert rel(r.X[:, i], ref["x"][9]) < 1e-10


def test_li_bicg_is_columnwise_bicg():
    """Sec. 2, Algorithm 1: column i of Li-BiCG is BiCG for A x_i = b_i."""
    A, B = problem(N=7, s=3, shift=0.3j)
    r = oracle.solve("li_bicg", A, B, tol=0.0, maxit=9)
    for i in range(3):
        ref = oracle.bicg_textbook(A, B[:, i], iters=9)
        assert rel(r.X[:, i], ref["x"][9]) < 1e-10


# ------------------------------------------------------------------------------------------
# Sec. 4: Bl-BiCG-rQ is Bl-BiCG (Eqs. (newalpha)-(newbetahat)); ||R|| = ||C||; phase invariance
# ------------------------------------------------------------------------------------------

def test_rq_equals_block_bicg():
    A, B = problem(N=12, s=3, shift=0.4j)
    for k in (1, 3, 8):
        a = oracle.solve("bl_bicg_rq", A, B, tol=0.0, maxit=k)
        b = oracle.solve("bl_bicg", A, B, tol=0.0, maxit=k)
        assert rel(a.X, b.X) < 1e-9


def test_rq_residual_norm_is_norm_of_C():
    A, B = problem(N=12, s=3, shift=0.4j)
    for k in (1, 4, 10):
        r = oracle.solve("bl_bicg_rq", A, B, tol=0.0, maxit=k)
        true = np.linalg.norm(B - A @ r.X) / np.linalg.norm(B)
        assert r.history[-1] == pytest.approx(true, rel=1e-8)


@pytest.mark.parametrize("pair", [("bl_bicg", "bl_bicg_rq"), ("bl_bicgstab", "bl_bicgstab_rq")])
@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_rq_survives_nearly_dependent_columns(pair, eps):
    """Sec. 4's motivation for the -rQ variants: when the columns of the block residual become
    (nearly) linearly dependent, the s x s matrices of the block method are (nearly) singular
    and it breaks down, while the variant that works with the QR factor Q of R converges.
    Here two pairs of right-hand sides differ by eps."""
    A, B = problem(N=16, pe=0.3, shift=0.3j, s=4, seed=2)
    rng = np.random.default_rng(0)
    B = B.copy()
    B[:, 1] = B[:, 0] + eps * (rng.standard_normal(B.shape[0]) + 1j * rng.standard_normal(B.shape[0]))
    B[:, 3] = B[:, 2] + eps * rng.standard_normal(B.shape[0])
    plain = oracle.solve(pair[0], A, B, tol=1e-8, maxit=300)
    rq = oracle.solve(pair[1], A, B, tol=1e-8, maxit=300)
    assert plain.status == Status.BREAKDOWN
    assert rq.status == Status.OK and rq.relres_true < 1e-7
    Xd = np.linalg.solve(A.toarray(), B)
    assert rel(rq.X, Xd) < 1e-5


def test_rq_invariant_under_qr_phase(monkeypatch):
    """X does not depend on the phases of the diagonal of the QR factors."""
    A, B = problem(N=10, s=3, shift=0.4j)
    ref = oracle.solve("bl_bicg_rq", A, B, tol=0.0, maxit=6)
    import oracle.methods as M

    def qr_other_phase(Z):
        Q, S = thin_qr(Z)
        ph = np.exp(1j * np.arange(1, Z.shape[1] + 1))
        return Q * ph[None, :], np.conj(ph)[:, None] * S

    monkeypatch.setattr(M, "thin_qr", qr_other_phase)
    alt = oracle.solve("bl_bicg_rq", A, B, tol=0.0, maxit=6)
    assert rel(alt.X, ref.X) < 1e-10


def test_stab_rq_equals_block_stab():
    A, B = problem(N=12, s=3, shift=0.4j)
    for k in (1, 3, 8):
        a = oracle.solve("bl_bicgstab_rq", A, B, tol=0.0, maxit=k)
        b = oracle.solve("bl_bicgstab", A, B, tol=0.0, maxit=k)
        assert rel(a.X, b.X) < 1e-9


def test_block_stab_krylov_space():
    """Bl-BiCGStab takes X_k from X_0 + K_{2k}(A, R_0) (Sec. 2)."""
    A, B = problem(N=8, s=2, shift=0.4j)
    Ad = A.toarray()
    for k in (1, 2):
        r = oracle.solve("bl_bicgstab", A, B, tol=0.0, maxit=k)
        K = np.hstack([np.linalg.matrix_power(Ad, j) @ B for j in range(2 * k)])
        Qk, _ = np.linalg.qr(K)
        assert np.linalg.norm(r.X - Qk @ (Qk.conj().T @ r.X)) < 1e-10 * np.linalg.norm(r.X)


def _stab_problem(kind):
    if kind == "convdiff":
        return problem(N=6, s=3, shift=0.3j)
    from workloads.random_csr import random_csr
    n = 40
    rp, ci, v = random_csr(n, max_row=5, seed=3, empty_frac=0.0)
    return oracle.csr_matrix_from_arrays(n, rp, ci, v), gaussian_block(n, 3, 5)


@pytest.mark.parametrize("method", ["bl_bicgstab", "bl_bicgstab_rq"])
@pytest.mark.parametrize("kind", ["convdiff", "complex"])
def test_block_stab_is_omega_polynomial_times_block_bicg(method, kind, monkeypatch):
    """Bl-BiCGStab of El Guennouni, Jbilou and Sadok (Sec. 2; the -rQ variant of Sec. 4 is the same
    method in exact arithmetic) at s > 1, from its defining property: after k steps
    R_k = Omega_k(A) R_k^BlBiCG with the scalar polynomial Omega_k(t) = prod_j (1 - omega_j t), where
    R_k^BlBiCG is the block-BiCG residual for the shadow block Rt_0 = R_0 (fixed here by brute-force
    Petrov-Galerkin, R_k^BlBiCG orthogonal to K_k(A^H, Rt_0)), and omega_k is the global
    steepest-descent step, the minimiser of ||(I - omega A) S_k||_F over omega for
    S_k = Omega_{k-1}(A) R_k^BlBiCG.  The omegas are recorded from the oracle's run; Omega_k(A)^{-1}
    R_k is formed by dense solves.  On the matrix with complex off-diagonal entries a transposed or
    unconjugated s x s solve anywhere in the recurrences breaks the identity at k >= 2."""
    import oracle.methods as M
    A, B = _stab_problem(kind)
    Ad = A.toarray()
    n = Ad.shape[0]
    I = np.eye(n)
    omegas = []
    name = "_omega" if method == "bl_bicgstab" else "_omega_weighted"
    orig = getattr(M, name)

    def recording(*args):
        w = orig(*args)
        omegas.append(complex(w))
        return w

    monkeypatch.setattr(M, name, recording)
    for k in (1, 2, 3, 4):
        omegas.clear()
        r = oracle.solve(method, A, B, tol=0.0, maxit=k)
        assert r.iters == k and len(omegas) == k
        Rk = B - Ad @ r.X
        R_bl = B - Ad @ _pg_iterate(Ad, B, B, k)
        Z = Rk
        for w in omegas:
            Z = np.linalg.solve(I - w * Ad, Z)
        assert rel(Z, R_bl) < 1e-9, (method, kind, k, rel(Z, R_bl))
        S = R_bl
        for w in omegas[:-1]:
            S = (I - w * Ad) @ S
        T = Ad @ S
        w_def = np.vdot(T, S) / np.vdot(T, T)  # argmin_w ||S - w T||_F
        assert abs(omegas[-1] - w_def) <= 1e-9 * abs(w_def), (method, kind, k)


# ------------------------------------------------------------------------------------------
# QMR: brute-force quasi-minimal residual from a dense bi-orthogonal basis (Sec. 2)
# ------------------------------------------------------------------------------------------

def _qmr_bruteforce(Ad, R0, Rh0, k):
    """Two-sided block Gram-Schmidt basis (full, not three-term) + least squares."""
    AH = Ad.conj().T
    V1, rho0 = thin_qr(R0)
    W1, _ = thin_qr(Rh0)
    Vs, Ws = [V1], [W1]
    for j in range(k):
        Vt = Ad @ Vs[-1]
        Wt = AH @ Ws[-1]
        for _ in range(2):  # oblique projections against all previous blocks, twice
            for Vi, Wi in zip(Vs, Ws):
                d = Wi.conj().T @ Vi
                Vt = Vt - Vi @ np.linalg.solve(d, Wi.conj().T @ Vt)
                Wt = Wt - Wi @ np.linalg.solve(d.conj().T, Vi.conj().T @ Wt)
        Vs.append(thin_qr(Vt)[0])
        Ws.append(thin_qr(Wt)[0])
    Vk = np.hstack(Vs[:k])
    Vk1 = np.hstack(Vs[: k + 1])
    Wk1 = np.hstack(Ws[: k + 1])
    T = np.linalg.solve(Wk1.conj().T @ Vk1, Wk1.conj().T @ (Ad @ Vk))
    s = R0.shape[1]
    E = np.zeros(((k + 1) * s, s), dtype=np.complex128)
    E[:s] = rho0
    Z = np.linalg.lstsq(T, E, rcond=None)[0]
    return Vk @ Z


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_block_qmr_quasi_minimal(k):
    A, B = problem(N=6, s=2, shift=0.3j)
    Ad = A.toarray()
    r = oracle.solve("bl_qmr", A, B, tol=0.0, maxit=k)
    assert rel(r.X, _qmr_bruteforce(Ad, B, B, k)) < 1e-9


@pytest.mark.parametrize("k", [2, 5, 8])
def test_block_qmr_quasi_minimal_random_shadow(k):
    """The left (shadow) recurrence only enters X through the bases; a random R^_0 exposes it."""
    A, B = problem(N=6, s=2, shift=0.3j)
    Rh0 = gaussian_block(B.shape[0], 2, 11)
    Ad = A.toarray()
    r = oracle.solve("bl_qmr", A, B, tol=0.0, maxit=k, shadow=Rh0)
    assert rel(r.X, _qmr_bruteforce(Ad, B, Rh0, k)) < 1e-9


@pytest.mark.parametrize("k", [2, 4])
def test_block_qmr_quasi_minimal_complex_offdiagonals(k):
    """Brute-force quasi-minimal residual iterate on a matrix with complex off-diagonals (the
    shadow side's A^H is only distinguishable from A^T on such a matrix)."""
    from workloads.random_csr import random_csr
    n = 30
    rp, ci, v = random_csr(n, max_row=5, seed=4, empty_frac=0.0)
    A = oracle.csr_matrix_from_arrays(n, rp, ci, v)
    B = gaussian_block(n, 2, 6)
    Rh0 = gaussian_block(n, 2, 7)
    r = oracle.solve("bl_qmr", A, B, tol=0.0, maxit=k, shadow=Rh0)
    assert rel(r.X, _qmr_bruteforce(A.toarray(), B, Rh0, k)) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_global_qmr_quasi_minimal(k):
    A, B = problem(N=6, s=2, shift=0.3j)
    K = kron_I(A, 2).toarray()
    r = oracle.solve("gl_qmr", A, B, tol=0.0, maxit=k)
    x_bf = _qmr_bruteforce(K, vec(B)[:, None], vec(B)[:, None], k)[:, 0]
    assert rel(vec(r.X), x_bf) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_li_qmr_is_columnwise_quasi_minimal(k):
    """Li-QMR (loop interchange, Sec. 2): column i after k steps is the quasi-minimal-residual
    iterate of the single system A x = b_i with shadow rh_i, built from a dense basis."""
    A, B = problem(N=6, s=3, shift=0.3j)
    Rh0 = gaussian_block(B.shape[0], 3, 17)
    Ad = A.toarray()
    r = oracle.solve("li_qmr", A, B, tol=0.0, maxit=k, shadow=Rh0)
    assert r.iters == k
    for i in range(3):
        x_bf = _qmr_bruteforce(Ad, B[:, i:i + 1], Rh0[:, i:i + 1], k)[:, 0]
        assert rel(r.X[:, i], x_bf) < 1e-9, i


def test_li_qmr_columns_are_independent():
    """Loop interchange: a column's iterates do not depend on the other columns (here: the
    same column solved alone, and the columns in reversed order)."""
    A, B = problem(N=8, s=3, shift=0.3j)
    r = oracle.solve("li_qmr", A, B, tol=0.0, maxit=7)
    alone = oracle.solve("li_qmr", A, B[:, 1:2], tol=0.0, maxit=7)
    rev = oracle.solve("li_qmr", A, B[:, ::-1].copy(), tol=0.0, maxit=7)
    assert rel(r.X[:, 1], alone.X[:, 0]) < 1e-13
    assert rel(r.X[:, ::-1], rev.X) < 1e-13


# ------------------------------------------------------------------------------------------
# recursive vs true residual, operation counts (Proposition 1), failure statuses
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("method", ALL)
def test_recursive_residual_matches_true(method):
    A, B = problem(N=10, s=3, shift=0.3j)
    for k in (1, 5, 12):
        r = oracle.solve(method, A, B, tol=0.0, maxit=k)
        true = np.linalg.norm(B - A @ r.X) / np.linalg.norm(B)
        assert abs(r.history[-1] - true) <= 1e-10


@pytest.mark.parametrize("method", ALL)
def test_matvec_counts(method):
    """Proposition 1: one A and one A^H block product per BiCG/QMR iteration (2s single
    matvecs); the economic methods apply A^H to one vector (s + 1); BiCGStab applies A twice."""
    A, B = problem(N=8, s=3)
    r = oracle.solve(method, A, B, tol=0.0, maxit=4)
    per = 4 if method.startswith("egl") else 6
    assert r.matvecs == per * r.iters


def test_status_breakdown_duplicate_columns():
    """Sec. 2: Bl-BiCG breaks down when an s x s matrix is singular (rank-deficient block)."""
    A, B = problem(N=8, s=3)
    B[:, 2] = B[:, 1]
    r = oracle.solve("bl_bicg", A, B, tol=1e-10, maxit=50)
    assert r.status == Status.BREAKDOWN


def test_status_nan_and_maxit_and_zero():
    A, B = problem(N=8, s=2)
    Bn = B.copy()
    Bn[3, 1] = np.nan
    assert oracle.solve("gl_bicg", A, Bn, tol=1e-10, maxit=10).status == Status.NAN
    assert oracle.solve("gl_bicg", A, B, tol=1e-14, maxit=3).status == Status.MAXIT
    z = oracle.solve("egl_bicg", A, np.zeros_like(B), tol=1e-10, maxit=10)
    assert z.status == Status.OK and z.iters == 0


def test_adjoint_identity():
    """<A x, y> = <x, A^H y> for the explicit adjoint used by every method."""
    A, B = problem(N=9, s=2)
    AH = oracle.adjoint(A)
    x, y = B[:, 0], B[:, 1]
    assert np.vdot(y, A @ x) == pytest.approx(np.vdot(AH @ y, x), rel=1e-13)


# ------------------------------------------------------------------------------------------
# Sec. 5 set-up: orthonormalised right-hand sides (B replaced by Q of B = Q S)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["egl_bicg", "gl_bicg", "bl_bicg", "bl_bicg_rq", "bl_bicgstab", "gl_qmr"])
def test_orthonormalized_rhs_gives_the_same_solution(method):
    """With orthonormalize_B the method runs on A Y = Q (B - A X_0 = Q S) and X = X_0 + Y S is
    returned: the same solution of A X = B, here against dense LU, from X_0 = 0 and from a
    non-zero X_0.  For the block methods the iterates themselves coincide with those of the plain
    run (the block Krylov spaces of R_0 and R_0 S^{-1} are equal and Bl-BiCG's Petrov-Galerkin
    conditions do not depend on the basis), which fixes that X = X_0 + Y S and not Y S^{-1}."""
    A, B = problem(N=8, s=3, shift=0.4j)
    Xd = np.linalg.solve(A.toarray(), B)
    X0 = 0.1 * gaussian_block(B.shape[0], 3, 7)
    for x0 in (None, X0):
        r = oracle.solve(method, A, B, X0=x0, tol=1e-12, maxit=400, orthonormalize_B=True)
        assert r.status == Status.OK, (method, r.status)
        assert rel(r.X, Xd) < 1e-9
        assert r.relres_true < 1e-10
    if method in ("bl_bicg", "bl_bicg_rq"):
        for k in (1, 2, 3):
            a = oracle.solve(method, A, B, tol=0.0, maxit=k, orthonormalize_B=True)
            b = oracle.solve(method, A, B, tol=0.0, maxit=k, shadow=None)
            # shadow: the plain run's default shadow is R_0, the orthonormalised run's is Q;
            # both span the same block Krylov spaces, so the Petrov-Galerkin iterate is the same
            assert rel(a.X, b.X) < 1e-9, (method, k)


def test_orthonormalized_rhs_rank_deficient_is_breakdown():
    A, B = problem(N=6, s=3, shift=0.4j)
    B = B.copy()
    B[:, 2] = B[:, 0]
    r = oracle.solve("gl_bicg", A, B, tol=1e-10, maxit=50, orthonormalize_B=True)
    assert r.status == Status.BREAKDOWN and r.breakdown_iter == 1 and r.iters == 0


def test_breakdown_iter_is_the_failing_iteration():
    """Duplicate right-hand sides make Bl-BiCG's first s x s matrix singular (Sec. 2)."""
    A, B = problem(N=6, s=3, shift=0.4j)
    B = B.copy()
    B[:, 2] = B[:, 1]
    r = oracle.solve("bl_bicg", A, B, tol=1e-10, maxit=50)
    assert r.status == Status.BREAKDOWN and r.breakdown_iter == r.iters + 1 == 1
    ok = oracle.solve("gl_bicg", A, B, tol=1e-10, maxit=200)
    assert ok.status == Status.OK and ok.breakdown_iter == 0
