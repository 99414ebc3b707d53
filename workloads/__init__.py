"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package builds the sparse operators and right-hand-side blocks that stand
in for the paper's experiments (Sec. 5, Examples 1-5).  It contains no step of
any Krylov method: only matrix entries, sparsity patterns and random numbers.

Layout conventions shared with every consumer:

* a sparse matrix is CSR: ``rowptr`` int64 (n+1), ``colidx`` int32 (nnz, sorted
  ascending within each row), ``vals`` complex128 (nnz);
* a block vector is a C-contiguous complex128 array of shape (n, s): row i holds
  the s entries of unknown i, i.e. the row-interleaved layout.
"""
from .stencil import ConvDiff, convdiff_csr, grid_nnz
from .rhs import gaussian_block, point_sources
from .lattice import Lattice4D, lattice_csr
from .random_csr import random_csr

__all__ = [
    "ConvDiff", "convdiff_csr", "grid_nnz",
    "gaussian_block", "point_sources",
    "Lattice4D", "lattice_csr", "random_csr",
]
