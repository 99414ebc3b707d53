"""Seeded random sparse matrices for kernel edge cases (empty rows, ragged row lengths)."""
from __future__ import annotations

import numpy as np


def random_csr(n: int, max_row: int = 9, seed: int = 0, real_offdiag: bool = False, empty_frac: float = 0.1,
               diag_shift: complex = 4.0 + 1.0j):
    """CSR (rowptr int64, colidx int32 sorted per row, vals complex128) of an n x n matrix.

    Row lengths are uniform in [0, max_row]; a fraction ``empty_frac`` of rows is
    empty apart from a diagonal entry (the diagonal is always stored, shifted by
    ``diag_shift`` so that the matrix is comfortably non-singular).  With
    ``real_offdiag`` every off-diagonal entry has a zero imaginary part.
    """
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        k = 0 if rng.random() < empty_frac else int(rng.integers(0, max_row + 1))
        c = set(rng.choice(n, size=min(k, n), replace=False).tolist()) if k else set()
        c.add(i)
        c = sorted(c)
        rows.extend([i] * len(c))
        cols.extend(c)
    rows = np.array(rows, dtype=np.int64)
    cols = np.array(cols, dtype=np.int32)
    vals = rng.standard_normal(len(cols)) + (0 if real_offdiag else 1j) * rng.standard_normal(len(cols))
    vals = vals.astype(np.complex128)
    vals[rows == cols] += diag_shift
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols, vals
