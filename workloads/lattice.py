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


# Lattice mass m.  With Haar-random links the spectrum's left edge on 4^4 lattices is at
# Re(lambda) ~ m + 2.03 (seed-to-seed spread ~0.05), and sigma_max / sigma_min reaches 1e3
# only at m ~ -2.05, where eigenvalues already lie in the left half-plane (on 16^4 all
# BiCG-type methods then fail).  Example 4's matrix has its spectrum in the right
# half-plane, so the mass keeps a margin: m = -1.8 (left edge +0.18, sigma_max / sigma_min
# = 54 on 4^4), from python -m workloads.calibrate_lattice (dense eigenvalues / SVD, CPU).
LATTICE_MASS = -1.8


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


def gamma5() -> np.ndarray:
    """gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 (Hermitian, anticommutes with every gamma_mu)."""
    return GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def lattice_csr(lat: Lattice4D, links: np.ndarray | None = None):
    """Assemble the lattice operator as CSR (rowptr int64, colidx int32, vals complex128).

    Only the 49 non-zeros of each row are generated: the diagonal, and for each of the
    8 hops the 2 spin columns of (I -+ gamma_mu) times the 3 colour columns of the link.
    """
    dims = tuple(int(L) for L in lat.dims)
    if min(dims) < 3:
        raise ValueError("every lattice extent must be >= 3 (forward and backward neighbours distinct)")
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
    cols = np.empty((sites, 4, 3, 49), dtype=np.int64)
    vals = np.empty((sites, 4, 3, 49), dtype=np.complex128)
    row_index = (site[:, None, None] * 4 + np.arange(4)[None, :, None]) * 3 + np.arange(3)[None, None, :]
    cols[..., 0] = row_index
    vals[..., 0] = 4.0 + lat.mass
    k = 1
    jj = np.arange(3)
    for mu in range(4):
        for step in (+1, -1):
            nb = shifted(mu, step)
            P = -0.5 * (eye - step * GAMMA[mu])
            if step > 0:
                U = links[mu]                                            # U_mu(x)
            else:
                U = np.conj(np.swapaxes(links[mu][nb], -1, -2))          # U_mu(x - mu)^H
            for a in range(4):
                bs = [b for b in range(4) if P[a, b] != 0]
                assert len(bs) == 2
                for t, b in enumerate(bs):
                    sl = slice(k + 3 * t, k + 3 * t + 3)
                    cols[:, a, :, sl] = ((nb * 4 + b) * 3)[:, None, None] + jj[None, None, :]
                    vals[:, a, :, sl] = P[a, b] * U
            k += 6
    assert k == 49
    cols = cols.reshape(n, 49)
    vals = vals.reshape(n, 49)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    rowptr = np.arange(0, 49 * (n + 1), 49, dtype=np.int64)
    return rowptr, cols.reshape(-1).astype(np.int32), np.ascontiguousarray(vals.reshape(-1))
