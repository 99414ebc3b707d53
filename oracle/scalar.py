"""Single right-hand-side textbook methods used to pin the simultaneous methods at s = 1.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 of the paper states that every simultaneous variant reduces to the
single-RHS method for s = 1.  These are the classical single-vector forms,
written in their usual textbook notation, independently of methods.py:

* BiCG (Fletcher): two-sided recurrences for r, rh, p, ph with scalar alpha, beta;
* BiCGStab (van der Vorst): rho_k = rt^H r_k, beta = (rho_k / rho_{k-1}) (alpha / omega).
"""
from __future__ import annotations

import numpy as np


def bicg_textbook(A, b, x0=None, rhat0=None, iters=10):
    """Run exactly ``iters`` BiCG steps; returns the list of iterates and residuals."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).reshape(-1).copy()
    AH = A.conj().T
    r = b - A @ x
    rh = r.copy() if rhat0 is None else np.asarray(rhat0, dtype=np.complex128).reshape(-1).copy()
    p, ph = r.copy(), rh.copy()
    rho = np.vdot(rh, r)
    xs, rs, rhs, ps, phs = [x.copy()], [r.copy()], [rh.copy()], [p.copy()], [ph.copy()]
    for _ in range(iters):
        q = A @ p
        qh = AH @ ph
        alpha = rho / np.vdot(ph, q)
        x = x + alpha * p
        r = r - alpha * q
        rh = rh - np.conj(alpha) * qh
        rho_new = np.vdot(rh, r)
        beta = rho_new / rho
        p = r + beta * p
        ph = rh + np.conj(beta) * ph
        rho = rho_new
        xs.append(x.copy())
        rs.append(r.copy())
        rhs.append(rh.copy())
        ps.append(p.copy())
        phs.append(ph.copy())
    return {"x": xs, "r": rs, "rh": rhs, "p": ps, "ph": phs}


def bicgstab_textbook(A, b, x0=None, rtilde=None, iters=10):
    """Run exactly ``iters`` BiCGStab steps (van der Vorst); returns iterates and residuals."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).reshape(-1).copy()
    r = b - A @ x
    rt = r.copy() if rtilde is None else np.asarray(rtilde, dtype=np.complex128).reshape(-1).copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    xs, rs = [x.copy()], [r.copy()]
    for _ in range(iters):
        rho = np.vdot(rt, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A @ p
        alpha = rho / np.vdot(rt, v)
        s = r - alpha * v
        t = A @ s
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        xs.append(x.copy())
        rs.append(r.copy())
    return {"x": xs, "r": rs}
