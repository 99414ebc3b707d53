"""Plain FP64 CPU oracle for the simultaneous short-recurrence Krylov methods.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it; the product package never does, and this package imports nothing
from the product package.  It shares no code with the CUDA path: the only
common inputs come from the ``workloads`` package (matrix entries and random
numbers, no method arithmetic).

Every method is written step by step in the paper's order and notation
(Rashedi, Birk, Frommer, Ebadi, "On short recurrence Krylov type methods for
linear systems with many right-hand sides"):

* Gl-BiCG      -- Sec. 2, Algorithm 2
* Bl-BiCG      -- Sec. 2, Algorithm 3 (adjoint re-use from the proof of Proposition 1)
* eGl-BiCG     -- Sec. 4, Algorithm 4
* Bl-BiCG-rQ   -- Sec. 4, Eqs. (QR), (newalpha)-(newbetahat), Algorithm 5
* Li-BiCG      -- Sec. 2, Algorithm 1
* Li-BiCGStab  -- the loop-interchange principle of Sec. 2 applied to BiCGStab
* Gl-BiCGStab, Bl-BiCGStab, Bl-BiCGStab-rQ, Gl-QMR, eGl-QMR, Bl-QMR -- named
  but not written out in the paper (Secs. 2 and 4); the readings implemented
  here are stated in each function's docstring.

Library primitives used as single steps: scipy.sparse CSR products, numpy
matrix products, LAPACK LU with partial pivoting (scipy.linalg.lu_factor) and
Householder QR (numpy.linalg.qr).

Pins (tests/test_oracle_*.py): dense LU solutions, textbook single-RHS
BiCG/BiCGStab at s=1, the Kronecker identity of the global methods (Sec. 2),
the identical-column shadow identity of the economic methods (Sec. 4),
brute-force Petrov-Galerkin and quasi-minimal-residual characterisations,
BiCG bi-orthogonality, recursive-vs-true residual agreement, the norm identity
||R|| = ||C|| of Sec. 4, and the rho values of Table 1.
"""
from .ops import (
    Status, adjoint, thin_qr, frob, trace_ip, sum_ip, gram, spmm, lu_solve,
    csr_matrix_from_arrays,
)
from .methods import (
    METHODS, solve, gl_bicg, egl_bicg, bl_bicg, bl_bicg_rq, li_bicg, li_bicgstab, li_qmr,
    gl_bicgstab, bl_bicgstab, bl_bicgstab_rq, gl_qmr, egl_qmr, bl_qmr,
)
from .scalar import bicg_textbook, bicgstab_textbook

__all__ = [
    "Status", "adjoint", "thin_qr", "frob", "trace_ip", "sum_ip", "gram", "spmm",
    "lu_solve", "csr_matrix_from_arrays", "METHODS", "solve",
    "gl_bicg", "egl_bicg", "bl_bicg", "bl_bicg_rq", "li_bicg", "li_bicgstab", "li_qmr",
    "gl_bicgstab", "bl_bicgstab", "bl_bicgstab_rq", "gl_qmr", "egl_qmr", "bl_qmr",
    "bicg_textbook", "bicgstab_textbook",
]
