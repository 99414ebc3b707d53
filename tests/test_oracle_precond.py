"""Pins of the ILU(0) right preconditioning of the oracle (CPU).

Sec. 5 repeats its experiments with an incomplete LU factorisation without fill-in as
right preconditioner.  The pins use what fixes ILU(0) independently of the oracle's
code: its defining identity (L U)_ij = A_ij on the pattern of A, the classical fact that
ILU(0) is the exact LU factorisation when the pattern admits no fill (tridiagonal, full),
and the preconditioned methods as the plain methods applied to the explicitly formed
dense matrix A M^{-1}.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import precond
from workloads import ConvDiff, convdiff_csr, gaussian_block, random_csr


def conv(dims, pe=0.4, shift=0.3j):
    op = ConvDiff(dims, tuple([pe] * len(dims)), shift)
    rp, ci, v = convdiff_csr(op)
    return oracle.csr_matrix_from_arrays(op.n, rp, ci, v)


@pytest.mark.parametrize("which", ["conv2d", "conv3d", "random"])
def test_ilu0_identity_on_the_pattern(which):
    if which == "conv2d":
        A = conv((12, 12))
    elif which == "conv3d":
        A = conv((6, 5, 4))
    else:
        rp, ci, v = random_csr(300, seed=4)
        A = oracle.csr_matrix_from_arrays(300, rp, ci, v)
    L, U = precond.ilu0(A)
    n = A.shape[0]
    assert np.all(sp.triu(L, 1).toarray() == 0) and np.allclose(L.diagonal(), 1)
    assert np.all(sp.tril(U, -1).toarray() == 0)
    LU = (L @ U).toarray()
    Ad = A.toarray()
    mask = Ad != 0
    assert np.max(np.abs(LU[mask] - Ad[mask])) <= 1e-12 * np.max(np.abs(Ad))
    # no fill: L and U live on the pattern of A
    assert np.all((L.toarray() != 0) <= (mask | np.eye(n, dtype=bool)))
    assert np.all((U.toarray() != 0) <= mask)


def test_ilu0_is_exact_lu_without_fill():
    """Tridiagonal (1D stencil) and full patterns admit no fill: ILU(0) = LU, M = A."""
    A = conv((40,))
    L, U = precond.ilu0(A)
    assert np.max(np.abs((L @ U - A).toarray())) <= 1e-13 * abs(A).max()
    rng = np.random.default_rng(2)
    D = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12)) + 30 * np.eye(12)
    L, U = precond.ilu0(sp.csr_matrix(D))
    assert np.max(np.abs((L @ U).toarray() - D)) <= 1e-12 * np.abs(D).max()


def test_exact_preconditioner_solves_in_one_iteration():
    """With M = A (tridiagonal case) A M^{-1} = I: one iteration gives X = A^{-1} B."""
    A = conv((50,))
    B = gaussian_block(50, 3, seed=1)
    L, U = precond.ilu0(A)
    res, X = precond.solve_right_preconditioned("gl_bicg", A, B, L, U, tol=1e-12, maxit=5)
    assert res.iters == 1
    assert np.linalg.norm(X - np.linalg.solve(A.toarray(), B)) <= 1e-12 * np.linalg.norm(X)


@pytest.mark.parametrize("method", ["gl_bicg", "bl_bicg", "egl_bicg", "bl_bicgstab", "gl_qmr", "li_bicg"])
def test_preconditioned_method_is_the_method_on_a_minv(method):
    """Right preconditioning only changes the operator: the residual history equals the plain
    method's on the dense matrix A M^{-1}, and X = M^{-1} Y."""
    A = conv((9, 8))
    n = A.shape[0]
    B = gaussian_block(n, 3, seed=2)
    L, U = precond.ilu0(A)
    res, X = precond.solve_right_preconditioned(method, A, B, L, U, tol=0.0, maxit=10)
    Minv = np.linalg.inv((L @ U).toarray())
    AM = A.toarray() @ Minv
    ref = oracle.solve(method, sp.csr_matrix(AM), B, tol=0.0, maxit=10)
    h, r = np.array(res.history), np.array(ref.history)
    assert len(h) == len(r)
    # relative agreement down to the rounding level of ||R_0|| (the histories reach 1e-19)
    assert np.all(np.abs(h - r) <= 1e-9 * r + 1e-14), np.max(np.abs(h - r) / (r + 1e-5))
    assert np.linalg.norm(X - Minv @ ref.X) <= 1e-9 * np.linalg.norm(X)


def test_apply_inverse_and_adjoint():
    A = conv((10, 7))
    L, U = precond.ilu0(A)
    V = gaussian_block(A.shape[0], 4, seed=3)
    M = (L @ U).toarray()
    assert np.linalg.norm(precond.apply_inverse(L, U, M @ V) - V) <= 1e-12 * np.linalg.norm(V)
    assert np.linalg.norm(precond.apply_inverse_adjoint(L, U, M.conj().T @ V) - V) <= 1e-12 * np.linalg.norm(V)


def test_ilu0_accelerates_convection_diffusion():
    """The effect Sec. 5 reports: fewer iterations with ILU(0) on convection-diffusion."""
    A = conv((24, 24), pe=0.5, shift=0.1j)
    B = gaussian_block(A.shape[0], 4, seed=0)
    plain = oracle.solve("egl_bicg", A, B, tol=1e-8, maxit=500)
    L, U = precond.ilu0(A)
    res, X = precond.solve_right_preconditioned("egl_bicg", A, B, L, U, tol=1e-8, maxit=500)
    assert res.status == oracle.Status.OK and plain.status == oracle.Status.OK
    assert res.iters < 0.6 * plain.iters, (res.iters, plain.iters)
    assert np.linalg.norm(B - A @ X) / np.linalg.norm(B) < 2e-8
