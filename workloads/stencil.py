"""Convection-diffusion operators on regular 2D/3D grids (Sec. 5, Examples 1-3).

The paper discretises -Laplace(u) + (convection) u = f with central finite
differences on an equispaced grid with Dirichlet boundaries (Example 1: 2D,
Example 2: 3D, 7 non-zeros per row).  The synthetic stand-ins use the same
pattern, written in the unscaled (multiplied by h^2) form:

* diagonal: 2*d + shift (shift is a complex number, e.g. 0.05i);
* neighbour at -1 along axis a: -1 - pe[a];
* neighbour at +1 along axis a: -1 + pe[a];

where pe[a] = v_a * h / 2 is the cell Peclet number of the convection velocity
v_a along axis a (central differences of v_a * du/dx_a times h^2).  Unknowns are
numbered with axis 0 fastest: i = x0 + N0*x1 + N0*N1*x2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class ConvDiff:
    """Parameters of a d-dimensional convection-diffusion stencil operator."""

    dims: tuple  # grid points per axis, axis 0 fastest
    pe: tuple  # cell Peclet number per axis
    shift: complex = 0.0

    @property
    def d(self) -> int:
        return len(self.dims)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    def strides(self):
        st, acc = [], 1
        for N in self.dims:
            st.append(acc)
            acc *= N
        return st

    def coefficients(self):
        """(centre, minus[a], plus[a]) stencil values as complex numbers."""
        centre = complex(2 * self.d) + complex(self.shift)
        minus = [complex(-1.0 - p) for p in self.pe]
        plus = [complex(-1.0 + p) for p in self.pe]
        return centre, minus, plus


def grid_nnz(dims) -> int:
    """Non-zeros of the (2d+1)-point Dirichlet stencil: (2d+1) n - 2 * sum_a n/N_a."""
    n = int(np.prod(dims))
    return (2 * len(dims) + 1) * n - 2 * sum(n // N for N in dims)


def convdiff_csr(op: ConvDiff, pe_override=None):
    """Assemble the stencil of ``op`` as CSR (rowptr int64, colidx int32, vals complex128).

    ``pe_override`` replaces ``op.pe`` (used when the Peclet numbers are learnable).
    """
    dims = tuple(int(N) for N in op.dims)
    d = len(dims)
    n = int(np.prod(dims))
    pe = op.pe if pe_override is None else pe_override
    centre = complex(2 * d) + complex(op.shift)
    strides = op.strides()
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for N in dims:
        coords.append(rem % N)
        rem //= N
    # offsets in ascending column order: -stride_{d-1}, ..., -stride_0, 0, +stride_0, ..., +stride_{d-1}
    cols, vals, masks = [], [], []
    for a in reversed(range(d)):
        cols.append(idx - strides[a])
        masks.append(coords[a] > 0)
        vals.append(complex(-1.0 - pe[a]))
    cols.append(idx)
    masks.append(np.ones(n, dtype=bool))
    vals.append(centre)
    for a in range(d):
        cols.append(idx + strides[a])
        masks.append(coords[a] < dims[a] - 1)
        vals.append(complex(-1.0 + pe[a]))
    C = np.stack(cols, axis=1)
    Mk = np.stack(masks, axis=1)
    V = np.broadcast_to(np.array(vals, dtype=np.complex128), C.shape)
    counts = Mk.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = C[Mk].astype(np.int32)
    values = np.ascontiguousarray(V[Mk])
    return rowptr, colidx, values


def convdiff_dpe_csr(op: ConvDiff, axis: int):
    """Derivative of the CSR values with respect to pe[axis] (same pattern as convdiff_csr).

    Entry (i, i - stride_axis) has derivative -1, entry (i, i + stride_axis) has +1,
    every other entry 0.
    """
    dims = tuple(int(N) for N in op.dims)
    d = len(dims)
    dpe = [0.0] * d
    zero = ConvDiff(dims, tuple(dpe), 0.0)
    rowptr, colidx, _ = convdiff_csr(zero)
    n = int(np.prod(dims))
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    st = zero.strides()[axis]
    out = np.zeros(colidx.shape[0], dtype=np.complex128)
    diff = colidx.astype(np.int64) - rows
    out[diff == -st] = -1.0
    out[diff == st] = 1.0
    return out
