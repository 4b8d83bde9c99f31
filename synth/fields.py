"""Seeded colour-vector sources on one parity of the lattice."""

import numpy as np


def parity_sites(dims, parity):
    """site_lex of the sites of a parity, in half-lattice index order i."""
    lx, ly, lz, lt = (int(d) for d in dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing='ij')
    lex = (x + lx * (y + ly * (z + lz * t))).ravel()
    par = ((x + y + z + t) & 1).ravel()
    return lex[par == parity]


def gaussian_source(vh, seed):
    """Complex Gaussian vector (vh, 3): re and im ~ N(0, 1), default_rng(seed).

    Draws ``standard_normal((vh, 3, 2))``: half-site index, colour, (re, im).
    """
    g = np.random.default_rng(seed).standard_normal((vh, 3, 2))
    return g[..., 0] + 1j * g[..., 1]


def gaussian_sources(vh, seeds):
    """Stack of Gaussian sources, shape (len(seeds), vh, 3)."""
    return np.stack([gaussian_source(vh, s) for s in seeds])
