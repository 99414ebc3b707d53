"""Calibration of the lattice mass m so that the operator's condition number is about 1e3.

Runs a dense SVD of the 4^4 x 12 operator (n = 3072) for a few masses and prints
sigma_max / sigma_min; the mass chosen from its output is LATTICE_MASS_KAPPA_1E3 in
lattice.py.  With Haar-random links the spectrum's lower edge sits near m = -2.4, and
the same m gives condition numbers of the same order on larger lattices of this
ensemble (the smallest singular value varies between configurations).

Usage: python -m workloads.calibrate_lattice
"""
import numpy as np
import scipy.sparse as sp

from .lattice import Lattice4D, lattice_csr


def kappa(L, m, seed=0):
    lat = Lattice4D((L,) * 4, m, seed)
    rp, ci, v = lattice_csr(lat)
    A = sp.csr_matrix((v, ci, rp), shape=(lat.n, lat.n)).toarray()
    sv = np.linalg.svd(A, compute_uv=False)
    return sv[0] / sv[-1]


if __name__ == "__main__":
    for m in (-2.2, -2.15, -2.1, -2.05, -2.0):
        print("m = %+.2f  kappa(4^4, seed 0) = %.3g" % (m, kappa(4, m)))
