"""Wilson-type nearest-neighbour operator on a periodic 4D lattice (Sec. 5, Example 4).

Example 4 of the paper uses a Wilson-Dirac matrix: 12 unknowns per lattice site
(4 spin x 3 colour), periodic nearest-neighbour couplings through a random
gauge field, 49 non-zeros per row.  The gauge configuration of the paper is not
available, so this module builds a synthetic stand-in with the same structure:

* unknown index (site*4 + spin)*3 + colour, site = x0 + L0*x1 + L0*L1*x2 + L0*L1*L2*x3;
* diagonal (4 + m) * I;
* forward hop x -> x+mu:  -1/2 (I - gamma_mu) (x) U_mu(x);
* backward hop x -> x-mu: -1/2 (I + gamma_mu) (x) U_mu(x-mu)^H;
* U_mu(x) in U(3) drawn from the Haar measure: Q of the QR factorisation of a
  complex Gaussian 3x3 matrix, with Q's columns multiplied by the phases of R's
  diagonal;
* gamma_mu: a fixed Hermitian, unitary set with one non-zero (+-1 or +-i) per
  row (chiral basis), so every (I +- gamma_mu) has two non-zeros per row and
  each row of the operator has 8*2*3 + 1 = 49 non-zeros.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# chiral-basis gamma matrices (Hermitian, square to I, pairwise anticommuting)
GAMMA = np.array(
    [
        [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
    ],
    dtype=np.complex128,
)


@dataclass(frozen=True)
class Lattice4D:
    dims: tuple  # (L0, L1, L2, L3), axis 0 fastest
    mass: float  # m in the diagonal 4 + m
    seed: int = 0

    @property
    def sites(self) -> int:
        return int(np.prod(self.dims))

    @property
    def n(self) -> int:
        return 12 * self.sites


def haar_links(dims, seed: int) -> np.ndarray:
    """Gauge links U[mu, site] in U(3), shape (4, sites, 3, 3), seeded PCG64."""
    sites = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((4, sites, 3, 3)) + 1j * rng.standard_normal((4, sites, 3, 3))
    Q, R = np.linalg.qr(Z)
    diag = np.diagonal(R, axis1=-2, axis2=-1)
    ph = diag / np.abs(diag)
    return Q * ph[..., None, :]


def lattice_csr(lat: Lattice4D, links: np.ndarray | None = None):
    """Assemble the lattice operator as CSR (rowptr int64, colidx int32, vals complex128)."""
    dims = tuple(int(L) for L in lat.dims)
    sites = int(np.prod(dims))
    n = 12 * sites
    if links is None:
        links = haar_links(dims, lat.seed)
    strides = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    site = np.arange(sites, dtype=np.int64)
    coords, rem = [], site.copy()
    for L in dims:
        coords.append(rem % L)
        rem //= L

    def shifted(mu, step):
        c = (coords[mu] + step) % dims[mu]
        return site + (c - coords[mu]) * strides[mu]

    eye = np.eye(4, dtype=np.complex128)
    # blocks[k]: (neighbour site array, 12x12 block per site) for the 9 couplings
    nbrs, blocks = [], []
    for mu in range(4):
        fwd = shifted(mu, +1)
        bwd = shifted(mu, -1)
        Pm = -0.5 * (eye - GAMMA[mu])
        Pp = -0.5 * (eye + GAMMA[mu])
        Uf = links[mu]  # U_mu(x)
        Ub = np.conj(np.swapaxes(links[mu][bwd], -1, -2))  # U_mu(x-mu)^H
        nbrs.append(fwd)
        blocks.append(np.einsum("ab,xij->xaibj", Pm, Uf).reshape(sites, 12, 12))
        nbrs.append(bwd)
        blocks.append(np.einsum("ab,xij->xaibj", Pp, Ub).reshape(sites, 12, 12))
    nbrs.append(site)
    blocks.append(np.broadcast_to((4.0 + lat.mass) * np.eye(12, dtype=np.complex128), (sites, 12, 12)))
    # gather all (row, col, val), drop structural zeros, sort rows and columns
    rows_l, cols_l, vals_l = [], [], []
    r12 = np.arange(12)
    for nb, blk in zip(nbrs, blocks):
        rr = (site[:, None, None] * 12 + r12[None, :, None]) + 0 * r12[None, None, :]
        cc = (nb[:, None, None] * 12 + r12[None, None, :]) + 0 * r12[None, :, None]
        mask = blk != 0
        rows_l.append(rr[mask])
        cols_l.append(cc[mask])
        vals_l.append(blk[mask])
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    vals = np.concatenate(vals_l)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    # merge duplicates (only possible when a dimension has extent <= 2)
    key = rows * n + cols
    uniq, start = np.unique(key, return_index=True)
    if uniq.shape[0] != key.shape[0]:
        vals = np.add.reduceat(vals, start)
        rows, cols = rows[start], cols[start]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols.astype(np.int32), np.ascontiguousarray(vals)
