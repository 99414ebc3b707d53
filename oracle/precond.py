"""ILU(0) right preconditioning for the simultaneous methods (Sec. 5, second set of experiments).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this package.

Sec. 5 repeats the experiments with an incomplete LU factorisation without fill-in as a
right preconditioner: A M^{-1} Y = B, X = M^{-1} Y, M = L U.  ILU(0) keeps the sparsity
pattern of A: L is unit lower triangular with the pattern of A's strictly lower part, U is
upper triangular with the pattern of A's upper part, and (L U)_ij = A_ij for every stored
(i, j).  The factorisation is the row-by-row (IKJ) Gaussian elimination restricted to
that pattern, written out with plain loops.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import LinearOperator, spsolve_triangular

from .ops import Breakdown


def ilu0(A):
    """ILU(0) of a square CSR matrix: returns (L, U) as CSR, L with unit diagonal (stored).

    Row i: for every stored k < i in increasing order, l_ik = a_ik / u_kk and, for every
    stored (k, j) with j > k that is also stored in row i, a_ij -= l_ik u_kj; the row's
    entries left of the diagonal are L's, the rest U's.  A zero pivot u_kk raises Breakdown.
    """
    A = sp.csr_matrix(A, dtype=np.complex128)
    A.sort_indices()
    n = A.shape[0]
    rp, ci = A.indptr, A.indices
    vals = A.data.copy()
    diag_pos = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            if ci[p] == i:
                diag_pos[i] = p
    if np.any(diag_pos < 0):
        raise Breakdown("ILU(0) needs every diagonal entry stored")
    pos = {}
    for i in range(n):
        pos.clear()
        for p in range(rp[i], rp[i + 1]):
            pos[int(ci[p])] = p
        for p in range(rp[i], rp[i + 1]):
            k = int(ci[p])
            if k >= i:
                break
            ukk = vals[diag_pos[k]]
            if ukk == 0:
                raise Breakdown("zero pivot in ILU(0)")
            lik = vals[p] / ukk
            vals[p] = lik
            for q in range(diag_pos[k] + 1, rp[k + 1]):
                j = int(ci[q])
                if j in pos:
                    vals[pos[j]] -= lik * vals[q]
    F = sp.csr_matrix((vals, ci.copy(), rp.copy()), shape=(n, n))
    L = sp.tril(F, k=-1, format="csr") + sp.identity(n, dtype=np.complex128, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L.tocsr(), U.tocsr()


def apply_inverse(L, U, V):
    """M^{-1} V = U^{-1} (L^{-1} V) by forward and backward substitution."""
    V = np.asarray(V, dtype=np.complex128)
    Z = spsolve_triangular(L, V, lower=True, unit_diagonal=True)
    return spsolve_triangular(U, Z, lower=False)


def apply_inverse_adjoint(L, U, W):
    """M^{-H} W = L^{-H} (U^{-H} W): U^H is lower, L^H unit upper triangular."""
    W = np.asarray(W, dtype=np.complex128)
    Z = spsolve_triangular(U.conj().T.tocsr(), W, lower=True)
    return spsolve_triangular(L.conj().T.tocsr(), Z, lower=False, unit_diagonal=True)


def solve_right_preconditioned(method, A, B, L, U, tol=1e-8, maxit=500, shadow=None):
    """Run ``method`` on A M^{-1} Y = B (Y_0 = 0) and return (Result, X = M^{-1} Y).

    The method sees the preconditioned operator through its products only: A M^{-1} V and
    (A M^{-1})^H W = M^{-H} A^H W.
    """
    from . import methods

    A = sp.csr_matrix(A, dtype=np.complex128)
    AH = A.conj().T.tocsr()
    n = A.shape[0]

    def mv(V):
        V = np.asarray(V)
        V2 = V.reshape(n, -1)
        return (A @ apply_inverse(L, U, V2)).reshape(V.shape)

    def rmv(W):
        W = np.asarray(W)
        W2 = W.reshape(n, -1)
        return apply_inverse_adjoint(L, U, AH @ W2).reshape(W.shape)

    Aop = LinearOperator((n, n), matvec=mv, matmat=mv, dtype=np.complex128)
    AHop = LinearOperator((n, n), matvec=rmv, matmat=rmv, dtype=np.complex128)
    res = methods.solve(method, Aop, B, tol=tol, maxit=maxit, shadow=shadow, AH=AHop)
    return res, apply_inverse(L, U, res.X)
