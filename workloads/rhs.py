"""Right-hand-side blocks (Sec. 5): seeded Gaussian blocks and unit-vector point sources."""
from __future__ import annotations

import numpy as np


def gaussian_block(n: int, s: int, seed: int = 0) -> np.ndarray:
    """(n, s) complex128 block with i.i.d. N(0,1) + i N(0,1) entries.

    Drawn from numpy's PCG64 generator seeded with ``seed``: first the (n, s)
    real parts, then the (n, s) imaginary parts.
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n, s))
    im = rng.standard_normal((n, s))
    out = np.empty((n, s), dtype=np.complex128)
    out.real = re
    out.imag = im
    return out


def point_sources(n: int, dofs_per_site: int, site: int, s: int | None = None) -> np.ndarray:
    """Unit vectors e_{site*dofs + j}, j = 0..s-1, as an (n, s) block.

    Example 4 of the paper solves for the 12 unit vectors belonging to the 12
    variables (spin x colour) of one lattice site.
    """
    if s is None:
        s = dofs_per_site
    B = np.zeros((n, s), dtype=np.complex128)
    base = site * dofs_per_site
    for j in range(s):
        B[base + j, j] = 1.0
    return B
