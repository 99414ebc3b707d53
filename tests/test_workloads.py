"""Structure of the seeded input generators (CPU): the stand-ins for the paper's examples."""
import numpy as np
import scipy.sparse as sp

from workloads import ConvDiff, Lattice4D, convdiff_csr, gaussian_block, grid_nnz, lattice_csr, point_sources
from workloads.lattice import GAMMA, gamma5, haar_links
from workloads.stencil import convdiff_dpe_csr


def test_gamma_matrices():
    I4 = np.eye(4)
    for mu in range(4):
        g = GAMMA[mu]
        assert np.allclose(g, g.conj().T)            # Hermitian
        assert np.allclose(g @ g, I4)                # squares to I
        assert np.all(np.count_nonzero(g, axis=1) == 1)
        for nu in range(mu + 1, 4):
            assert np.allclose(g @ GAMMA[nu] + GAMMA[nu] @ g, 0)   # anticommute
    g5 = gamma5()
    assert np.allclose(g5, g5.conj().T) and np.allclose(g5 @ g5, I4)


def test_links_are_unitary():
    U = haar_links((3, 3, 3, 3), 1)
    eye = np.eye(3)
    assert np.allclose(np.einsum("msij,mskj->msik", U, U.conj()), eye)


def test_lattice_gamma5_hermiticity_and_pattern():
    """The Wilson-type operator satisfies gamma5 A gamma5 = A^H (forward/backward hops consistent)."""
    lat = Lattice4D((4, 3, 5, 3), mass=-0.3, seed=2)
    rp, ci, v = lattice_csr(lat)
    n = lat.n
    assert np.all(np.diff(rp) == 49)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    G5 = sp.kron(sp.identity(n // 12), sp.kron(sp.csr_matrix(gamma5()), sp.identity(3)))
    assert abs(A.conj().T - G5 @ A @ G5).max() < 1e-14
    assert np.allclose(A.diagonal(), 4.0 - 0.3)
    # free field (all links = I): momentum-zero constant spinor fields are eigenvectors with eigenvalue m
    Ufree = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, lat.sites, 3, 3)).copy()
    rp0, ci0, v0 = lattice_csr(lat, links=Ufree)
    A0 = sp.csr_matrix((v0, ci0, rp0), shape=(n, n))
    x = np.tile(np.arange(1, 13, dtype=np.complex128), lat.sites)
    assert np.allclose(A0 @ x, -0.3 * x)


def test_convdiff_pattern_and_derivative():
    op = ConvDiff((5, 4, 3), (0.3, -0.2, 0.1), 0.05j)
    rp, ci, v = convdiff_csr(op)
    assert len(v) == grid_nnz(op.dims)
    A = sp.csr_matrix((v, ci, rp), shape=(op.n, op.n)).toarray()
    # interior row: centre 6 + shift, neighbours -1 -+ pe along each axis
    i = 1 + 5 * (1 + 4 * 1)
    assert A[i, i] == 6 + 0.05j
    assert A[i, i - 1] == -1 - 0.3 and A[i, i + 1] == -1 + 0.3
    assert A[i, i - 20] == -1 - 0.1 and A[i, i + 20] == -1 + 0.1
    # values are affine in pe with the stated derivative pattern
    for a in range(3):
        pe = list(op.pe)
        pe[a] += 0.5
        _, _, v2 = convdiff_csr(op, pe_override=pe)
        assert np.allclose((v2 - v) / 0.5, convdiff_dpe_csr(op, a))


def test_rhs_generators():
    B = gaussian_block(100, 3, seed=4)
    assert B.shape == (100, 3) and B.dtype == np.complex128 and B.flags.c_contiguous
    assert np.array_equal(B, gaussian_block(100, 3, seed=4))
    P = point_sources(12 * 10, 12, site=7)
    assert np.array_equal(P[84:96], np.eye(12))
