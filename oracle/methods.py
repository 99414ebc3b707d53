"""The simultaneous Krylov methods, step by step, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Common driver conventions (Sec. 5, first paragraph): the initial guess X0
(default 0), the initial shadow residual R^(0)^ = R^(0) for the block and global
methods and r^(0)^ = arithmetic mean of the columns of R^(0) for the economic
methods, and the stopping test ||R^(k)||_F <= tol * ||R^(0)||_F on the
recursively updated residual (for the -rQ variants ||C^(k)||_F, which equals
||R^(k)||_F by the norm remark after Algorithm 5).

Failure rules (readings; the paper only says "breaks down"):
* a scalar quotient num/den breaks down when den == 0 or |den| <= eps |num|;
* an s x s solve breaks down when an LU pivot satisfies |u_ii| <= 64 eps ||M||_F;
* a relative residual above 1e8 stops the iteration as DIVERGED, a non-finite
  one as NAN; at the end a true relative residual above 1 turns MAXIT into
  DIVERGED ("div." in Table 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .ops import (
    Breakdown, Status, adjoint, check_scalar, frob, gram, lu_solve, spmm, sum_ip,
    thin_qr, trace_ip, upper_right_solve,
)


@dataclass
class Result:
    X: np.ndarray
    status: Status
    iters: int
    matvecs: int
    history: list = field(default_factory=list)  # ||R_k||/||R_0|| for k = 0..iters
    relres_true: float = float("nan")  # ||B - A X||_F / ||R_0||_F at exit
    breakdown_iter: int = 0  # BREAKDOWN: the iteration (iters + 1) that could not be completed; else 0


class _Monitor:
    """Iteration counter and stopping test shared by all methods."""

    def __init__(self, tol, maxit):
        self.tol = float(tol)
        self.maxit = int(maxit)
        self.iters = 0
        self.matvecs = 0
        self.history = []
        self.status = Status.MAXIT
        self.done = False
        self.X = None

    def begin(self, nrm0):
        self.nrm0 = float(nrm0)
        self.history.append(1.0)
        if not np.isfinite(self.nrm0):
            self.status, self.done = Status.NAN, True
        elif self.nrm0 == 0.0:
            self.status, self.done = Status.OK, True
        elif self.maxit <= 0:
            self.status, self.done = Status.MAXIT, True

    def step(self, rnorm):
        """Record ||R_k|| after one iteration; returns True when the iteration must stop."""
        self.iters += 1
        rel = float(rnorm) / self.nrm0
        self.history.append(rel)
        if not np.isfinite(rel):
            self.status, self.done = Status.NAN, True
        elif rel <= self.tol:
            self.status, self.done = Status.OK, True
        elif rel > 1e8:
            self.status, self.done = Status.DIVERGED, True
        elif self.iters >= self.maxit:
            self.status, self.done = Status.MAXIT, True
        return self.done


# --------------------------------------------------------------------------------------
# BiCG family
# --------------------------------------------------------------------------------------

def li_bicg(A, AH, B, X0, Rh0, mon):
    """Li-BiCG, Sec. 2, Algorithm 1: s BiCG iterations with diagonal alpha, beta."""
    s = B.shape[1]
    X = X0.copy()
    R = B - spmm(A, X)
    Rh = R.copy() if Rh0 is None else Rh0.copy()
    P, Ph = R.copy(), Rh.copy()
    mon.X = X
    mon.begin(frob(R))
    rho = np.array([np.vdot(Rh[:, i], R[:, i]) for i in range(s)])  # <r_i, rh_i> = rh_i^H r_i
    while not mon.done:
        Q = spmm(A, P)
        alpha = np.array([check_scalar(rho[i], np.vdot(Ph[:, i], Q[:, i])) for i in range(s)])
        X = X + P * alpha[None, :]
        R = R - Q * alpha[None, :]
        Rh = Rh - spmm(AH, Ph) * np.conj(alpha)[None, :]
        mon.matvecs += 2 * s
        mon.X = X
        if mon.step(frob(R)):
            break
        rho_new = np.array([np.vdot(Rh[:, i], R[:, i]) for i in range(s)])
        beta = np.array([check_scalar(rho_new[i], rho[i]) for i in range(s)])
        P = R + P * beta[None, :]
        Ph = Rh + Ph * np.conj(beta)[None, :]
        rho = rho_new
    return X


def gl_bicg(A, AH, B, X0, Rh0, mon):
    """Gl-BiCG, Sec. 2, Algorithm 2: BiCG for (I (x) A) x = b with <X, Y> = tr(Y^H X)."""
    X = X0.copy()
    R = B - spmm(A, X)
    Rh = R.copy() if Rh0 is None else Rh0.copy()
    P, Ph = R.copy(), Rh.copy()
    mon.X = X
    mon.begin(frob(R))
    rho = trace_ip(Rh, R)  # tr(Rh^H R)
    while not mon.done:
        Q = spmm(A, P)
        alpha = check_scalar(rho, trace_ip(Ph, Q))
        X = X + alpha * P
        R = R - alpha * Q
        Rh = Rh - np.conj(alpha) * spmm(AH, Ph)
        mon.matvecs += 2 * B.shape[1]
        mon.X = X
        if mon.step(frob(R)):
            break
        rho_new = trace_ip(Rh, R)
        beta = check_scalar(rho_new, rho)
        P = R + beta * P
        Ph = Rh + np.conj(beta) * Ph
        rho = rho_new
    return X


def egl_bicg(A, AH, B, X0, rh0, mon):
    """eGl-BiCG, Sec. 4, Algorithm 4: Gl-BiCG with the single shadow vector rh (R^ = rh 1^T).

    Uses tr(1 rh^H R) = sum(rh^H R) (Sec. 4); A^H multiplies one n-vector per iteration.
    """
    X = X0.copy()
    R = B - spmm(A, X)
    rh = R.mean(axis=1) if rh0 is None else np.asarray(rh0).reshape(-1).copy()
    P, ph = R.copy(), rh.copy()
    mon.X = X
    mon.begin(frob(R))
    rho = sum_ip(rh, R)
    while not mon.done:
        Q = spmm(A, P)
        alpha = check_scalar(rho, sum_ip(ph, Q))
        X = X + alpha * P
        R = R - alpha * Q
        rh = rh - np.conj(alpha) * spmm(AH, ph[:, None])[:, 0]
        mon.matvecs += B.shape[1] + 1
        mon.X = X
        if mon.step(frob(R)):
            break
        rho_new = sum_ip(rh, R)
        beta = check_scalar(rho_new, rho)
        P = R + beta * P
        ph = rh + np.conj(beta) * ph
        rho = rho_new
    return X


def bl_bicg(A, AH, B, X0, Rh0, mon):
    """Bl-BiCG, Sec. 2, Algorithm 3 (O'Leary's block BiCG).

    As in the proof of Proposition 1, (P^H Qh) is taken as (Ph^H Q)^H and
    (R^H Rh) as (Rh^H R)^H, and Rh^H R is carried over from the previous iteration.
    """
    X = X0.copy()
    R = B - spmm(A, X)
    Rh = R.copy() if Rh0 is None else Rh0.copy()
    P, Ph = R.copy(), Rh.copy()
    mon.X = X
    mon.begin(frob(R))
    G = gram(Rh, R)  # (Rh^(k))^H R^(k)
    while not mon.done:
        Q = spmm(A, P)
        Qh = spmm(AH, Ph)
        M = gram(Ph, Q)  # (Ph^(k))^H Q^(k)
        alpha = lu_solve(M, G)
        alpha_h = lu_solve(M.conj().T, G.conj().T)
        X = X + P @ alpha
        R = R - Q @ alpha
        Rh = Rh - Qh @ alpha_h
        mon.matvecs += 2 * B.shape[1]
        mon.X = X
        if mon.step(frob(R)):
            break
        G_new = gram(Rh, R)
        beta = lu_solve(G, G_new)
        beta_h = lu_solve(G.conj().T, G_new.conj().T)
        P = R + P @ beta
        Ph = Rh + Ph @ beta_h
        G = G_new
    return X


def bl_bicg_rq(A, AH, B, X0, Rh0, mon):
    """Bl-BiCG-rQ, Sec. 4, Algorithm 5: block BiCG on QR factors R = Q C, Rh = Qh Ch.

    alpha, alpha_h, beta, beta_h are the right-hand sides of Eqs. (newalpha)-(newbetahat);
    (V^H Wh) is taken as (Vh^H W)^H and (Q^H Qh) as (Qh^H Q)^H.  The loop starts
    at index 0 (the algorithm's initialisation).
    """
    X = X0.copy()
    R = B - spmm(A, X)
    Rh = R.copy() if Rh0 is None else Rh0.copy()
    Q, C = thin_qr(R)
    Qh, Ch = thin_qr(Rh)
    V, Vh = Q.copy(), Qh.copy()
    mon.X = X
    mon.begin(frob(C))
    G = gram(Qh, Q)  # (Qh^(k))^H Q^(k)
    while not mon.done:
        W = spmm(A, V)
        Wh = spmm(AH, Vh)
        M = gram(Vh, W)  # (Vh^(k))^H W^(k)
        alpha = lu_solve(M, G)
        alpha_h = lu_solve(M.conj().T, G.conj().T)
        X = X + V @ (alpha @ C)
        Q_new, S = thin_qr(Q - W @ alpha)
        C = S @ C
        Qh_new, Sh = thin_qr(Qh - Wh @ alpha_h)
        Ch = Sh @ Ch
        mon.matvecs += 2 * B.shape[1]
        mon.X = X
        if mon.step(frob(C)):
            break
        G_new = gram(Qh_new, Q_new)
        beta = lu_solve(G, Sh.conj().T @ G_new)
        beta_h = lu_solve(G.conj().T, S.conj().T @ G_new.conj().T)
        V = Q_new + V @ beta
        Vh = Qh_new + Vh @ beta_h
        Q, Qh, G = Q_new, Qh_new, G_new
    return X


# --------------------------------------------------------------------------------------
# BiCGStab family (not written out in the paper; Sec. 2 and Sec. 4)
# --------------------------------------------------------------------------------------

def _omega(T, S):
    """Steepest-descent step omega = tr(T^H S) / tr(T^H T); 0 if T == 0 (then S == 0 too)."""
    tt = trace_ip(T, T)
    ts = trace_ip(T, S)
    if not (np.isfinite(tt) and np.isfinite(ts)):
        raise FloatingPointError("non-finite omega")
    if tt == 0:
        return 0.0
    return ts / tt


def _omega_weighted(Tp, Sp, C):
    """omega of Bl-BiCGStab-rQ: tr(T'^H S' C C^H) / tr(T'^H T' C C^H), which is omega = tr(T^H S) /
    tr(T^H T) of Bl-BiCGStab for S = S' C, T = T' C; 0 if the denominator vanishes."""
    CC = C @ C.conj().T
    num = np.trace(gram(Tp, Sp) @ CC)
    den = np.trace(gram(Tp, Tp) @ CC)
    if not (np.isfinite(num) and np.isfinite(den)):
        raise FloatingPointError("non-finite omega")
    return 0.0 if den == 0 else num / den


def gl_bicgstab(A, AH, B, X0, Rt0, mon):
    """Gl-BiCGStab: van der Vorst's BiCGStab for (I (x) A) x = b with <X, Y> = tr(Y^H X).

    Reading of Sec. 2 (global principle) and Sec. 3 (Gl-BiCGStab of Jbilou et al.):
      V = A P; alpha = tr(Rt^H R) / tr(Rt^H V); S = R - alpha V; T = A S;
      omega = tr(T^H S) / tr(T^H T); X += alpha P + omega S; R = S - omega T;
      beta = (tr(Rt^H R_new) / tr(Rt^H R)) (alpha / omega); P = R + beta (P - omega V).
    """
    X = X0.copy()
    R = B - spmm(A, X)
    Rt = R.copy() if Rt0 is None else Rt0.copy()
    P = R.copy()
    mon.X = X
    mon.begin(frob(R))
    rho = trace_ip(Rt, R)
    while not mon.done:
        V = spmm(A, P)
        alpha = check_scalar(rho, trace_ip(Rt, V))
        S = R - alpha * V
        T = spmm(A, S)
        omega = _omega(T, S)
        X = X + alpha * P + omega * S
        R = S - omega * T
        mon.matvecs += 2 * B.shape[1]
        mon.X = X
        if mon.step(frob(R)):
            break
        rho_new = trace_ip(Rt, R)
        beta = check_scalar(rho_new, rho) * check_scalar(alpha, omega)
        P = R + beta * (P - omega * V)
        rho = rho_new
    return X


def li_bicgstab(A, AH, B, X0, Rt0, mon):
    """Li-BiCGStab: the loop-interchange principle of Sec. 2 (Algorithm 1) applied to BiCGStab.

    s independent BiCGStab iterations sharing the block products A P and A S:
      V = A P; alpha_i = rho_i / (rt_i^H v_i); S = R - V diag(alpha); T = A S;
      omega_i = (t_i^H s_i) / (t_i^H t_i); X += P diag(alpha) + S diag(omega);
      R = S - T diag(omega); beta_i = (rho_new_i / rho_i)(alpha_i / omega_i);
      P = R + (P - V diag(omega)) diag(beta).
    """
    s = B.shape[1]
    X = X0.copy()
    R = B - spmm(A, X)
    Rt = R.copy() if Rt0 is None else Rt0.copy()
    P = R.copy()
    mon.X = X
    mon.begin(frob(R))
    rho = np.array([np.vdot(Rt[:, i], R[:, i]) for i in range(s)])
    while not mon.done:
        V = spmm(A, P)
        alpha = np.array([check_scalar(rho[i], np.vdot(Rt[:, i], V[:, i])) for i in range(s)])
        S = R - V * alpha[None, :]
        T = spmm(A, S)
        omega = np.zeros(s, dtype=np.complex128)
        for i in range(s):
            tt = np.vdot(T[:, i], T[:, i])
            ts = np.vdot(T[:, i], S[:, i])
            if not (np.isfinite(tt) and np.isfinite(ts)):
                raise FloatingPointError("non-finite omega")
            omega[i] = 0.0 if tt == 0 else ts / tt
        X = X + P * alpha[None, :] + S * omega[None, :]
        R = S - T * omega[None, :]
        mon.matvecs += 2 * s
        mon.X = X
        if mon.step(frob(R)):
            break
        rho_new = np.array([np.vdot(Rt[:, i], R[:, i]) for i in range(s)])
        beta = np.array([check_scalar(rho_new[i], rho[i]) * check_scalar(alpha[i], omega[i]) for i in range(s)])
        P = R + (P - V * omega[None, :]) * beta[None, :]
        rho = rho_new
    return X


def bl_bicgstab(A, AH, B, X0, Rt0, mon):
    """Bl-BiCGStab (El Guennouni, Jbilou, Sadok), reading of Sec. 2:

      V = A P; (Rt^H V) alpha = Rt^H R; S = R - V alpha; T = A S;
      omega = tr(T^H S) / tr(T^H T)   (the "global" steepest-descent step);
      X += P alpha + omega S; R = S - omega T;
      (Rt^H V) beta = -Rt^H T; P = R + (P - omega V) beta.
    """
    X = X0.copy()
    R = B - spmm(A, X)
    Rt = R.copy() if Rt0 is None else Rt0.copy()
    P = R.copy()
    mon.X = X
    mon.begin(frob(R))
    while not mon.done:
        V = spmm(A, P)
        M = gram(Rt, V)
        alpha = lu_solve(M, gram(Rt, R))
        S = R - V @ alpha
        T = spmm(A, S)
        omega = _omega(T, S)
        X = X + P @ alpha + omega * S
        R = S - omega * T
        mon.matvecs += 2 * B.shape[1]
        mon.X = X
        if mon.step(frob(R)):
            break
        beta = lu_solve(M, -gram(Rt, T))
        P = R + (P - omega * V) @ beta
    return X


def bl_bicgstab_rq(A, AH, B, X0, Rt0, mon):
    """Bl-BiCGStab-rQ: Bl-BiCGStab on the QR factors R = Q C, P = V C (Sec. 4, last remark).

    Derived as Algorithm 5 is derived from Algorithm 3:
      W = A V; alpha = (Rt^H W)^{-1} (Rt^H Q); S' = Q - W alpha; T' = A S';
      omega = tr(T'^H S' C C^H) / tr(T'^H T' C C^H)   (= omega of Bl-BiCGStab);
      X += (V alpha + omega S') C;  S' - omega T' = Q_new Sigma;  C_new = Sigma C;
      V_new = Q_new + (V - omega W) beta Sigma^{-1},  beta = -(Rt^H W)^{-1} (Rt^H T').
    The stopping test uses ||C||_F.
    """
    X = X0.copy()
    R = B - spmm(A, X)
    Rt = R.copy() if Rt0 is None else Rt0.copy()
    Q, C = thin_qr(R)
    V = Q.copy()
    mon.X = X
    mon.begin(frob(C))
    while not mon.done:
        W = spmm(A, V)
        M = gram(Rt, W)
        alpha = lu_solve(M, gram(Rt, Q))
        Sp = Q - W @ alpha
        Tp = spmm(A, Sp)
        omega = _omega_weighted(Tp, Sp, C)
        X = X + (V @ alpha + omega * Sp) @ C
        Q_new, Sig = thin_qr(Sp - omega * Tp)
        C = Sig @ C
        mon.matvecs += 2 * B.shape[1]
        mon.X = X
        if mon.step(frob(C)):
            break
        beta = lu_solve(M, -gram(Rt, Tp))
        d = np.abs(np.diag(Sig))
        if np.any(d <= 64.0 * np.finfo(float).eps * np.linalg.norm(Sig)):
            raise Breakdown("rank-deficient residual block")
        V = Q_new + upper_right_solve((V - omega * W) @ beta, Sig)
        Q = Q_new
    return X


# --------------------------------------------------------------------------------------
# QMR family (not written out in the paper; Sec. 2 and Sec. 4)
# --------------------------------------------------------------------------------------

def _givens(a, b):
    """Complex Givens rotation G = [[c, s], [-conj(s), c]] with G [a; b] = [r; 0], c real >= 0."""
    if b == 0:
        return 1.0, 0.0, a
    if a == 0:
        return 0.0, 1.0, b
    nu = np.hypot(abs(a), abs(b))
    ph = a / abs(a)
    return abs(a) / nu, ph * np.conj(b) / nu, ph * nu


def _glqmr_core(A, AH, B, X0, Wfirst, mon, w_is_vector):
    """QMR without look-ahead on (I (x) A) with the trace inner product (Gl-QMR / eGl-QMR).

    Two-sided Lanczos with unit Frobenius norm basis blocks:
      V_1 = R_0 / rho_1, W_1 = Rh_0 / xi_1, delta_k = tr(W_k^H V_k),
      A V_k = V_{k+1} rho_{k+1} + V_k alpha_k + V_{k-1} beta_k,
      alpha_k = tr(W_k^H A V_k) / delta_k, beta_k = xi_k delta_k / delta_{k-1},
      A^H W_k = W_{k+1} xi_{k+1} + W_k conj(alpha_k) + W_{k-1} gamma_k,
      gamma_k = conj(rho_k delta_k / delta_{k-1}).
    X_k = X_0 + [V_1..V_k] z_k with z_k minimising || rho_1 e_1 - T_{k+1,k} z ||_2,
    solved by complex Givens rotations; X and R follow from the search directions
    D_k = (V_k - u_{k-2,k} D_{k-2} - u_{k-1,k} D_{k-1}) / u_kk and A D_k (same recurrence on A V_k).

    For eGl-QMR (Sec. 4) W_k = w_k 1^T is held as the single vector w_k:
    tr(W^H Y) = sum(w^H Y), A^H W = (A^H w) 1^T, ||W||_F = sqrt(s) ||w||.
    """
    s = B.shape[1]
    X = X0.copy()
    R = B - spmm(A, X)
    if w_is_vector:
        W = R.mean(axis=1) if Wfirst is None else np.asarray(Wfirst).reshape(-1).copy()

        def ip(w, Y):
            return sum_ip(w, Y)

        def wnorm(w):
            return np.sqrt(s) * frob(w)

        def adj(w):
            return spmm(AH, w[:, None])[:, 0]
    else:
        W = R.copy() if Wfirst is None else Wfirst.copy()
        ip = trace_ip
        wnorm = frob

        def adj(Wb):
            return spmm(AH, Wb)
    mon.X = X
    mon.begin(frob(R))
    if mon.done:
        return X
    rho_k = frob(R)
    xi_k = wnorm(W)
    if xi_k == 0:
        raise Breakdown("zero shadow residual")
    V = R / rho_k
    W = W / xi_k
    V_prev = np.zeros_like(V)
    W_prev = np.zeros_like(W)
    delta = ip(W, V)
    delta_prev = None
    t = complex(rho_k)  # current entry of the rotated right-hand side rho_1 e_1
    rot1 = rot2 = None  # Givens rotations of steps k-1 and k-2
    D1 = np.zeros_like(V)
    D2 = np.zeros_like(V)
    AD1 = np.zeros_like(V)
    AD2 = np.zeros_like(V)
    k = 0
    while not mon.done:
        k += 1
        if delta == 0 or not np.isfinite(delta):
            raise Breakdown("Lanczos breakdown: delta_k = 0")
        Y = spmm(A, V)
        Yh = adj(W)
        alpha = ip(W, Y) / delta
        if k >= 2:
            beta = xi_k * delta / delta_prev
            gamma = np.conj(rho_k * delta / delta_prev)
        else:
            beta = gamma = 0.0
        Vt = Y - alpha * V - beta * V_prev
        Wt = Yh - np.conj(alpha) * W - gamma * W_prev
        rho_next = frob(Vt)
        xi_next = wnorm(Wt)
        # column k of T_{k+1,k}: (beta_k, alpha_k, rho_{k+1}) in rows k-1, k, k+1
        u2, u1, u0 = 0.0, beta, alpha
        if rot2 is not None:
            c, sn = rot2
            u2, u1 = sn * u1, c * u1
        if rot1 is not None:
            c, sn = rot1
            u1, u0 = c * u1 + sn * u0, -np.conj(sn) * u1 + c * u0
        c, sn, ukk = _givens(u0, rho_next)
        if ukk == 0:
            raise Breakdown("singular tridiagonal")
        tau = c * t
        t = -np.conj(sn) * t
        D = (V - u2 * D2 - u1 * D1) / ukk
        AD = (Y - u2 * AD2 - u1 * AD1) / ukk
        X = X + tau * D
        R = R - tau * AD
        mon.matvecs += s + (1 if w_is_vector else s)
        mon.X = X
        D2, D1 = D1, D
        AD2, AD1 = AD1, AD
        rot2, rot1 = rot1, (c, sn)
        if mon.step(frob(R)):
            break
        if rho_next == 0 or xi_next == 0:
            raise Breakdown("invariant subspace reached with non-zero residual")
        V_prev, W_prev = V, W
        V = Vt / rho_next
        W = Wt / xi_next
        delta_prev, delta = delta, ip(W, V)
        rho_k, xi_k = rho_next, xi_next
    return X


def li_qmr(A, AH, B, X0, Rh0, mon):
    """Li-QMR: the loop-interchanged QMR of Sec. 2 (the paper names the Li variants of its three
    families; Algorithm 1 shows the construction for BiCG).  The s scalar QMR iterations (no
    look-ahead) on A x_i = b_i with shadow rh_i run in lockstep, one step of every column per
    iteration; the iteration stops on ||R||_F.  Per column i:
      v_1 = r_0 / rho_1, w_1 = rh_0 / xi_1, delta_k = w_k^H v_k,
      alpha_k = w_k^H A v_k / delta_k, beta_k = xi_k delta_k / delta_{k-1},
      gamma_k = conj(rho_k delta_k / delta_{k-1}),
      A v_k = v_{k+1} rho_{k+1} + alpha_k v_k + beta_k v_{k-1},
      A^H w_k = w_{k+1} xi_{k+1} + conj(alpha_k) w_k + gamma_k w_{k-1},
    the tridiagonal least-squares problem by complex Givens rotations, and
    d_k = (v_k - u_{k-2,k} d_{k-2} - u_{k-1,k} d_{k-1}) / u_kk, x += tau_k d_k, r -= tau_k A d_k.
    """
    s = B.shape[1]
    X = X0.copy()
    R = B - spmm(A, X)
    W = R.copy() if Rh0 is None else Rh0.copy()
    mon.X = X
    mon.begin(frob(R))
    if mon.done:
        return X
    rho_k = np.linalg.norm(R, axis=0)
    xi_k = np.linalg.norm(W, axis=0)
    if np.any(xi_k == 0) or np.any(rho_k == 0):
        raise Breakdown("zero column residual or shadow")
    V = R / rho_k[None, :]
    W = W / xi_k[None, :]
    V_prev = np.zeros_like(V)
    W_prev = np.zeros_like(W)

    def cdot(U, Y):  # column-wise u_i^H y_i
        return np.einsum("ij,ij->j", U.conj(), Y)

    delta = cdot(W, V)
    delta_prev = None
    t = rho_k.astype(np.complex128)
    rot1 = rot2 = None  # per-column Givens rotations (c, s) of steps k-1 and k-2
    D1 = np.zeros_like(V)
    D2 = np.zeros_like(V)
    AD1 = np.zeros_like(V)
    AD2 = np.zeros_like(V)
    k = 0
    while not mon.done:
        k += 1
        if np.any(delta == 0) or not np.all(np.isfinite(delta)):
            raise Breakdown("Lanczos breakdown: delta_k = 0 in a column")
        Y = spmm(A, V)
        Yh = spmm(AH, W)
        alpha = cdot(W, Y) / delta
        if k >= 2:
            beta = xi_k * delta / delta_prev
            gamma = np.conj(rho_k * delta / delta_prev)
        else:
            beta = gamma = np.zeros(s, dtype=np.complex128)
        Vt = Y - V * alpha[None, :] - V_prev * beta[None, :]
        Wt = Yh - W * np.conj(alpha)[None, :] - W_prev * gamma[None, :]
        rho_next = np.linalg.norm(Vt, axis=0)
        xi_next = np.linalg.norm(Wt, axis=0)
        u2 = np.zeros(s, dtype=np.complex128)
        u1 = beta.astype(np.complex128)
        u0 = alpha.astype(np.complex128)
        if rot2 is not None:
            c, sn = rot2
            u2, u1 = sn * u1, c * u1
        if rot1 is not None:
            c, sn = rot1
            u1, u0 = c * u1 + sn * u0, -np.conj(sn) * u1 + c * u0
        cs = np.zeros(s)
        sns = np.zeros(s, dtype=np.complex128)
        ukk = np.zeros(s, dtype=np.complex128)
        for i in range(s):
            cs[i], sns[i], ukk[i] = _givens(u0[i], rho_next[i])
        if np.any(ukk == 0):
            raise Breakdown("singular tridiagonal in a column")
        tau = cs * t
        t = -np.conj(sns) * t
        D = (V - D2 * u2[None, :] - D1 * u1[None, :]) / ukk[None, :]
        AD = (Y - AD2 * u2[None, :] - AD1 * u1[None, :]) / ukk[None, :]
        X = X + D * tau[None, :]
        R = R - AD * tau[None, :]
        mon.matvecs += 2 * s
        mon.X = X
        D2, D1 = D1, D
        AD2, AD1 = AD1, AD
        rot2, rot1 = rot1, (cs, sns)
        if mon.step(frob(R)):
            break
        if np.any(rho_next == 0) or np.any(xi_next == 0):
            raise Breakdown("invariant subspace reached in a column")
        V_prev, W_prev = V, W
        V = Vt / rho_next[None, :]
        W = Wt / xi_next[None, :]
        delta_prev, delta = delta, cdot(W, V)
        rho_k, xi_k = rho_next, xi_next
    return X


def gl_qmr(A, AH, B, X0, Rh0, mon):
    """Gl-QMR: QMR (no look-ahead) for (I (x) A) x = b with <X, Y> = tr(Y^H X) (Sec. 2)."""
    return _glqmr_core(A, AH, B, X0, Rh0, mon, w_is_vector=False)


def egl_qmr(A, AH, B, X0, rh0, mon):
    """eGl-QMR (Sec. 4): Gl-QMR with the identical-column shadow block W = w 1^T."""
    return _glqmr_core(A, AH, B, X0, rh0, mon, w_is_vector=True)


def bl_qmr(A, AH, B, X0, Rh0, mon):
    """Bl-QMR with block products, without look-ahead or deflation (reading of Sec. 2).

    Block two-sided Lanczos with orthonormal basis blocks:
      R_0 = V_1 rho_0, Rh_0 = W_1 xi_1 (thin QR), delta_k = W_k^H V_k,
      A V_k = V_{k+1} rho_{k+1} + V_k alpha_k + V_{k-1} beta_k,
      alpha_k = delta_k^{-1} W_k^H A V_k, beta_k = delta_{k-1}^{-1} xi_k^H delta_k,
      A^H W_k = W_{k+1} xi_{k+1} + W_k alpha^_k + W_{k-1} beta^_k,
      alpha^_k = delta_k^{-H} (W_k^H A V_k)^H, beta^_k = delta_{k-1}^{-H} rho_k^H delta_k^H,
    with V_{k+1} rho_{k+1} and W_{k+1} xi_{k+1} thin QR factorisations.
    X_k = X_0 + [V_1..V_k] Z_k, Z_k minimising || E_1 rho_0 - T_{k+1,k} Z ||_F, via
    2s x 2s unitary block rotations (complete QR of the 2s x s block column);
    D_k = (V_k - D_{k-2} U_{k-2,k} - D_{k-1} U_{k-1,k}) U_kk^{-1}, X += D_k tau_k,
    R -= (A D_k) tau_k.
    """
    s = B.shape[1]
    X = X0.copy()
    R = B - spmm(A, X)
    Rh = R.copy() if Rh0 is None else Rh0.copy()
    mon.X = X
    mon.begin(frob(R))
    if mon.done:
        return X
    V, rho0 = thin_qr(R)
    W, xi_k = thin_qr(Rh)
    rho_k = rho0
    V_prev = np.zeros_like(V)
    W_prev = np.zeros_like(W)
    delta = gram(W, V)
    delta_prev = None
    t = rho0.copy()  # current s x s block of the rotated right-hand side E_1 rho_0
    om1 = om2 = None  # 2s x 2s unitaries of steps k-1 and k-2
    Z = np.zeros((s, s), dtype=np.complex128)
    D1 = np.zeros_like(V)
    D2 = np.zeros_like(V)
    AD1 = np.zeros_like(V)
    AD2 = np.zeros_like(V)
    k = 0
    while not mon.done:
        k += 1
        Y = spmm(A, V)
        Yh = spmm(AH, W)
        WY = gram(W, Y)
        alpha = lu_solve(delta, WY)
        alpha_h = lu_solve(delta.conj().T, WY.conj().T)
        if k >= 2:
            beta = lu_solve(delta_prev, xi_k.conj().T @ delta)
            beta_h = lu_solve(delta_prev.conj().T, rho_k.conj().T @ delta.conj().T)
        else:
            beta = beta_h = Z
        Vt = Y - V @ alpha - V_prev @ beta
        Wt = Yh - W @ alpha_h - W_prev @ beta_h
        V_next, rho_next = thin_qr(Vt)
        W_next, xi_next = thin_qr(Wt)
        # block column k of T_{k+1,k}: (beta_k, alpha_k, rho_{k+1}) in block rows k-1, k, k+1
        u2, u1, u0 = Z, beta, alpha
        if om2 is not None:
            tmp = om2 @ np.vstack([Z, u1])
            u2, u1 = tmp[:s], tmp[s:]
        if om1 is not None:
            tmp = om1 @ np.vstack([u1, u0])
            u1, u0 = tmp[:s], tmp[s:]
        Qf, Rf = np.linalg.qr(np.vstack([u0, rho_next]), mode="complete")
        om = Qf.conj().T
        Ukk = Rf[:s, :s]
        if np.any(np.abs(np.diag(Ukk)) <= 64.0 * np.finfo(float).eps * max(np.linalg.norm(Ukk), 1e-300)):
            raise Breakdown("singular block tridiagonal")
        tt = om @ np.vstack([t, Z])
        tau, t = tt[:s], tt[s:]
        D = upper_right_solve(V - D2 @ u2 - D1 @ u1, Ukk)
        AD = upper_right_solve(Y - AD2 @ u2 - AD1 @ u1, Ukk)
        X = X + D @ tau
        R = R - AD @ tau
        mon.matvecs += 2 * s
        mon.X = X
        D2, D1 = D1, D
        AD2, AD1 = AD1, AD
        om2, om1 = om1, om
        if mon.step(frob(R)):
            break
        V_prev, W_prev = V, W
        V, W = V_next, W_next
        delta_prev, delta = delta, gram(W, V)
        rho_k, xi_k = rho_next, xi_next
    return X


# --------------------------------------------------------------------------------------
# driver
# --------------------------------------------------------------------------------------

METHODS = {
    "bl_bicg": bl_bicg,
    "bl_bicg_rq": bl_bicg_rq,
    "gl_bicg": gl_bicg,
    "egl_bicg": egl_bicg,
    "bl_bicgstab": bl_bicgstab,
    "bl_bicgstab_rq": bl_bicgstab_rq,
    "gl_bicgstab": gl_bicgstab,
    "bl_qmr": bl_qmr,
    "gl_qmr": gl_qmr,
    "egl_qmr": egl_qmr,
    "li_bicg": li_bicg,
    "li_bicgstab": li_bicgstab,
    "li_qmr": li_qmr,
}


def solve(method, A, B, X0=None, tol=1e-8, maxit=500, shadow=None, AH=None, orthonormalize_B=False):
    """Run ``method`` on A X = B; returns a Result.

    ``shadow``: initial shadow residual block (n x s) for the block/global
    methods, or the single shadow vector (n) for the economic methods; None
    selects the paper's defaults (R_0, or the mean of R_0's columns).

    ``orthonormalize_B``: the set-up of Sec. 5, in which the right-hand sides are
    replaced by the orthonormal factor Q of their thin QR decomposition.  With an
    initial guess: R_0 = B - A X_0 = Q S, the method solves A Y = Q from Y = 0, and
    X = X_0 + Y S.  The history and the stopping test refer to the system with Q,
    relres_true to A X = B.
    """
    B = np.asarray(B, dtype=np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    X0 = np.zeros_like(B) if X0 is None else np.asarray(X0, dtype=np.complex128).copy()
    if AH is None:
        AH = adjoint(A)
    if orthonormalize_B:
        R0 = B - spmm(A, X0)
        nrm0 = frob(R0)
        if nrm0 == 0.0 or not np.isfinite(nrm0):
            st = Status.OK if nrm0 == 0.0 else Status.NAN
            return Result(X=X0, status=st, iters=0, matvecs=0, history=[1.0], relres_true=nrm0)
        Q, S = thin_qr(R0)
        d = np.abs(np.diag(S))
        if np.any(d <= 64.0 * np.finfo(float).eps * np.linalg.norm(S)):  # numerically rank deficient
            return Result(X=X0, status=Status.BREAKDOWN, iters=0, matvecs=0, history=[1.0], relres_true=1.0,
                          breakdown_iter=1)
        r = solve(method, A, Q, None, tol=tol, maxit=maxit, shadow=shadow, AH=AH)
        X = X0 + r.X @ S
        r.X = X
        r.relres_true = float(frob(B - spmm(A, X)) / nrm0)
        if r.status == Status.MAXIT and r.relres_true > 1.0:
            r.status = Status.DIVERGED
        return r
    fn = METHODS[method]
    mon = _Monitor(tol, maxit)
    mon.X = X0
    with np.errstate(all="ignore"):
        try:
            X = fn(A, AH, B, X0, shadow, mon)
        except Breakdown:
            mon.status = Status.BREAKDOWN
            X = mon.X
        except FloatingPointError:
            mon.status = Status.NAN
            X = mon.X
        R = B - spmm(A, X)
        nrm0 = getattr(mon, "nrm0", frob(B - spmm(A, X0)))
        rel = frob(R) / nrm0 if nrm0 > 0 else frob(R)
    status = mon.status
    if status == Status.MAXIT and rel > 1.0:
        status = Status.DIVERGED
    if not np.isfinite(rel) and status != Status.BREAKDOWN:
        status = Status.NAN
    return Result(X=X, status=status, iters=mon.iters, matvecs=mon.matvecs, history=mon.history,
                  relres_true=float(rel), breakdown_iter=mon.iters + 1 if status == Status.BREAKDOWN else 0)
