"""Building blocks of the oracle: block products, inner products, small dense solves, thin QR.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation (Sec. 1 and Sec. 2 of the paper): block vectors are n x s complex
matrices; the global inner product is <X, Y> = tr(Y^H X) (Sec. 2, Eq. (global));
the economic methods use sum(r^H R), the sum of the entries of the row vector
r^H R (Sec. 4, before Algorithm 4).
"""
from __future__ import annotations

import enum

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps


class Status(enum.IntEnum):
    """Outcome of a solve (same numbering as the C interface's kr_status)."""

    OK = 0  # converged: ||R_k||_F <= tol * ||R_0||_F
    BREAKDOWN = 1  # a scalar denominator vanished or an s x s matrix was singular
    DIVERGED = 2  # residual grew beyond 1e8 * ||R_0||, or final true residual > ||R_0||
    NAN = 3  # a non-finite value appeared
    MAXIT = 4  # iteration limit reached without convergence


class Breakdown(Exception):
    pass


def csr_matrix_from_arrays(n, rowptr, colidx, vals):
    """scipy CSR matrix from the (rowptr, colidx, vals) arrays of the workloads package."""
    return sp.csr_matrix((np.asarray(vals, dtype=np.complex128), np.asarray(colidx), np.asarray(rowptr)),
                         shape=(n, n))


def adjoint(A):
    """A^H as an explicit CSR matrix (conjugate transpose)."""
    return A.conj().T.tocsr()


def spmm(A, V):
    """Matrix-block-vector product A V (Sec. 1): one sparse product for all s columns."""
    return np.asarray(A @ V)


def gram(U, V):
    """s x s (or 1 x s) matrix U^H V."""
    return np.conj(U).T @ V


def trace_ip(U, V):
    """tr(U^H V) = sum_ij conj(U_ij) V_ij (global inner product <V, U>, Sec. 2)."""
    return complex(np.vdot(U, V))


def sum_ip(u, V):
    """sum(u^H V) for a single n-vector u and an n x s block V (Sec. 4)."""
    return complex(np.sum(np.conj(u) @ V))


def frob(X):
    """Frobenius norm."""
    return float(np.linalg.norm(X))


def check_scalar(num, den):
    """Breakdown rule for a scalar quotient num/den: den == 0, |den| <= eps*|num|, or non-finite."""
    if not (np.isfinite(num) and np.isfinite(den)):
        raise FloatingPointError("non-finite coefficient")
    if den == 0 or abs(den) <= EPS * abs(num):
        raise Breakdown("scalar denominator vanished")
    return num / den


def lu_solve(M, N):
    """M^{-1} N by LU with partial pivoting; breakdown if a pivot |u_ii| <= 64 eps ||M||_F."""
    M = np.asarray(M, dtype=np.complex128)
    N = np.asarray(N, dtype=np.complex128)
    if not (np.all(np.isfinite(M)) and np.all(np.isfinite(N))):
        raise FloatingPointError("non-finite s x s matrix")
    lu, piv = sla.lu_factor(M, check_finite=False)
    tolp = 64.0 * EPS * np.linalg.norm(M)
    if np.any(np.abs(np.diag(lu)) <= tolp):
        raise Breakdown("singular s x s matrix")
    return sla.lu_solve((lu, piv), N, check_finite=False)


def thin_qr(Z):
    """Thin QR  Z = Q S  with Q^H Q = I and S upper triangular with real diagonal >= 0 (Sec. 4, Eq. (QR)).

    Householder QR (LAPACK) followed by the diagonal phase normalisation that
    makes the factorisation unique for full-rank Z.
    """
    Q, S = np.linalg.qr(Z, mode="reduced")
    d = np.diag(S)
    ph = np.ones_like(d)
    nz = d != 0
    ph[nz] = d[nz] / np.abs(d[nz])
    Q = Q * ph[None, :]
    S = np.conj(ph)[:, None] * S
    return Q, S


def upper_right_solve(Y, S):
    """Y S^{-1} for upper triangular S."""
    # (Y S^{-1})^T = S^{-T} Y^T: solve the lower triangular system S^T Z = Y^T
    Z = sla.solve_triangular(S.T, Y.T, lower=True)
    return Z.T
