"""Calibration of the lattice mass m (LATTICE_MASS in lattice.py).

Runs a dense eigenvalue decomposition and SVD of the 4^4 x 12 operator (n = 3072) for a
few masses and seeds, and prints the spectrum's left edge min Re(lambda) and
sigma_max / sigma_min.  The mass is chosen so that the spectrum stays in the right
half-plane with a margin (as for the Wilson matrix of Example 4), at the largest
condition number that margin allows.

Usage: python -m workloads.calibrate_lattice
"""
import numpy as np
import scipy.sparse as sp

from .lattice import Lattice4D, lattice_csr


def edge_and_kappa(L, m, seed=0):
    lat = Lattice4D((L,) * 4, m, seed)
    rp, ci, v = lattice_csr(lat)
    A = sp.csr_matrix((v, ci, rp), shape=(lat.n, lat.n)).toarray()
    ev = np.linalg.eigvals(A)
    sv = np.linalg.svd(A, compute_uv=False)
    return ev.real.min(), sv[0] / sv[-1]


if __name__ == "__main__":
    for m in (-2.05, -2.0, -1.95, -1.9, -1.85, -1.8):
        for seed in (0, 1):
            e, k = edge_and_kappa(4, m, seed)
            print("m = %+.2f seed %d  min Re(lambda) = %+.3f  kappa = %.3g" % (m, seed, e, k))
