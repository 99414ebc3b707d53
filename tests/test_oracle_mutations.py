"""Planted mistakes in the oracle, each caught by the pins (CPU only).

The pins in test_oracle_pins.py check the oracle against facts that do not
come from the oracle itself: dense LU, the classical single-RHS methods, the
Kronecker form of the global methods (Sec. 2), brute-force Petrov-Galerkin and
quasi-minimal-residual solutions, and exact identities between methods.  Here
each test plants one plausible mistake in the oracle: a dropped conjugate, a
transposed coefficient matrix or factor, swapped operands, or a wrong rotation.
It then checks that at least one of the named pins fails.  A pin set that let
a mistake through would not pin the oracle.  The mistakes are planted with
pytest's monkeypatch, on the CPU, in the oracle's module namespace only; the
single-RHS textbook methods the pins compare against are not touched.
"""
import numpy as np
import pytest

import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

import oracle.methods as M
from oracle import precond as P
from oracle.ops import lu_solve as _lu_solve, thin_qr as _thin_qr

import test_oracle_pins as pins
import test_oracle_precond as ppins


def _omega_swapped(T, S):
    return M.__dict__["_omega_orig"](S, T)


class _BetaSolveTransposed:
    """lu_solve with its matrix transposed whenever it receives the same matrix object twice in a
    row.  Bl-BiCGStab and Bl-BiCGStab-rQ are the only methods whose beta solve reuses the alpha
    solve's matrix (Rt^H V, resp. Rt^H W), so this plants a transposed beta solve in both
    variants alike: a reading error the two would share, invisible at s = 1."""

    def __init__(self):
        self.last = None

    def __call__(self, Mx, N):
        same = Mx is self.last
        self.last = Mx
        return _lu_solve(np.asarray(Mx).T if same else Mx, N)


def _givens_sign_flipped(a, b):
    """The complex Givens rotation with the sign of its off-diagonal entry flipped, so that it
    no longer annihilates b."""
    if b == 0:
        return 1.0, 0.0, a
    if a == 0:
        return 0.0, 1.0, b
    nu = np.hypot(abs(a), abs(b))
    ph = a / abs(a)
    return abs(a) / nu, -ph * np.conj(b) / nu, ph * nu


def _minv_wrong_order(L, U, V):
    """L^{-1} (U^{-1} V) instead of U^{-1} (L^{-1} V)."""
    Z = spsolve_triangular(U, np.asarray(V, dtype=np.complex128), lower=False)
    return spsolve_triangular(L, Z, lower=True, unit_diagonal=True)


def _mhinv_no_conj(L, U, W):
    """M^{-T} W instead of M^{-H} W."""
    Z = spsolve_triangular(U.T.tocsr(), np.asarray(W, dtype=np.complex128), lower=True)
    return spsolve_triangular(L.T.tocsr(), Z, lower=False, unit_diagonal=True)


def _ilu0_conj_pivots(A):
    """ILU(0) with the diagonal of U conjugated."""
    L, U = P.__dict__["ilu0_orig"](A)
    d = U.diagonal()
    return L, (U - sp.diags(d) + sp.diags(np.conj(d))).tocsr()


def _stab_pin(method):
    """The Omega-polynomial pin of Bl-BiCGStab on the complex matrix, with its own monkeypatch."""
    def run():
        with pytest.MonkeyPatch.context() as mp:
            pins.test_block_stab_is_omega_polynomial_times_block_bicg(method, "complex", mp)
    return run


# name -> (module, attribute, replacement, pins that must not all pass)
MUTATIONS = {
    # Sec. 2, Algorithm 3: the s x s matrices are Ph^H Q and Rh^H R
    "gram without conjugate": (M, "gram", lambda U, V: np.asarray(U).T @ V,
                               [lambda: pins.test_block_bicg_petrov_galerkin("bl_bicg")]),
    # Sec. 2, Eq. (global): <X, Y> = tr(Y^H X)
    "trace inner product without conjugate": (
        M, "trace_ip", lambda U, V: complex(np.sum(np.asarray(U) * np.asarray(V))),
        [pins.test_global_bicg_is_kron_bicg, pins.test_global_bicgstab_is_kron_bicgstab,
         pins.test_global_qmr_is_kron_qmr]),
    # Sec. 4, Algorithm 4: sum(r^H R)
    "economic sum without conjugate": (
        M, "sum_ip", lambda u, V: complex(np.sum(np.asarray(u) @ V)),
        [lambda: pins.test_economic_equals_global_with_identical_columns(("egl_bicg", "gl_bicg"))]),
    # Algorithm 3: alpha = (Ph^H Q)^{-1} (Rh^H R), not its transpose
    "coefficient solve with transposed matrix": (
        M, "lu_solve", lambda Mx, N: _lu_solve(np.asarray(Mx).T, N),
        [lambda: pins.test_block_bicg_petrov_galerkin("bl_bicg")]),
    "coefficient solve with conjugated matrix": (
        M, "lu_solve", lambda Mx, N: _lu_solve(np.conj(Mx), N),
        [lambda: pins.test_block_bicg_petrov_galerkin("bl_bicg")]),
    # Sec. 4, Eq. (QR): Z = Q S with S upper triangular (a transposed factor breaks C_{k+1} = S C_k)
    "thin QR returns the transposed factor": (
        M, "thin_qr", lambda Z: (lambda QS: (QS[0], QS[1].T))(_thin_qr(Z)),
        [lambda: pins.test_block_bicg_petrov_galerkin("bl_bicg_rq"), pins.test_rq_equals_block_bicg]),
    # BiCGStab: omega = tr(T^H S) / tr(T^H T)
    "omega with swapped operands": (
        M, "_omega", _omega_swapped,
        [pins.test_global_bicgstab_is_kron_bicgstab, lambda: pins.test_s1_reduces_to_bicgstab("bl_bicgstab")]),
    # Bl-BiCGStab at s > 1 (Sec. 2, El Guennouni-Jbilou-Sadok): (Rt^H V) beta = -Rt^H T, shared by
    # the -rQ variant; caught by the Omega-polynomial pin without the s = 1 or rQ-equality pins
    "beta solve transposed in both block BiCGStab variants": (
        M, "lu_solve", _BetaSolveTransposed(),
        [_stab_pin("bl_bicgstab"), _stab_pin("bl_bicgstab_rq")]),
    # the shadow recurrences multiply by A^H, not A^T (distinguishable only with complex
    # off-diagonal entries: for a complex shift of a real matrix both give the same Krylov spaces)
    "adjoint without conjugate": (
        M, "adjoint", lambda A: A.T.tocsr(),
        [lambda: pins.test_block_bicg_petrov_galerkin_complex_offdiagonals("bl_bicg"),
         lambda: pins.test_block_qmr_quasi_minimal_complex_offdiagonals(4)]),
    # QMR: the complex Givens rotation that annihilates the subdiagonal entry
    "Givens rotation with flipped sign": (
        M, "_givens", _givens_sign_flipped,
        [lambda: pins.test_global_qmr_quasi_minimal(3), lambda: pins.test_global_qmr_quasi_minimal(4)]),
    # Sec. 5, ILU(0) right preconditioning: M^{-1} = U^{-1} L^{-1}, M^{-H} = L^{-H} U^{-H}
    "preconditioner factors applied in the wrong order": (
        P, "apply_inverse", _minv_wrong_order,
        [ppins.test_apply_inverse_and_adjoint, lambda: ppins.test_preconditioned_method_is_the_method_on_a_minv("gl_bicg")]),
    "adjoint preconditioner without conjugate": (
        P, "apply_inverse_adjoint", _mhinv_no_conj,
        [ppins.test_apply_inverse_and_adjoint, lambda: ppins.test_preconditioned_method_is_the_method_on_a_minv("gl_bicg")]),
    "ILU(0) pivots conjugated": (
        P, "ilu0", _ilu0_conj_pivots,
        [lambda: ppins.test_ilu0_identity_on_the_pattern("conv2d")]),
}


def _fails(pin):
    try:
        pin()
    except (AssertionError, ArithmeticError, np.linalg.LinAlgError):
        return True
    except Exception as e:  # a breakdown raised by the planted mistake also counts as caught
        return type(e).__name__ in ("Breakdown",)
    return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    mod, attr, bad, pin_set = MUTATIONS[name]
    assert hasattr(mod, attr), attr
    if attr in ("_omega", "ilu0"):  # the replacement calls the original
        monkeypatch.setitem(mod.__dict__, attr + "_orig", getattr(mod, attr))
    monkeypatch.setattr(mod, attr, bad)
    caught = [_fails(p) for p in pin_set]
    assert any(caught), "planted mistake '%s' passed every pin in its set" % name


def test_pin_sets_pass_without_mistakes():
    """The same pin sets pass on the unmodified oracle (so a caught mistake is the mistake's doing)."""
    seen = set()
    for _, _, _, pin_set in MUTATIONS.values():
        for p in pin_set:
            if id(p) in seen:
                continue
            seen.add(id(p))
            assert not _fails(p)
