"""Seeded inputs of the NPR four-fermion workload (Eq. 1).

Propagators are Gaussian complex 3 x 3 matrices per site, ``[site][colour]
[source colour]``, standing in for the momentum-source quark propagators of
the paper's NPR code (which need a lattice and an inverter we do not ship as
data).  The operator list is the B_K basis of one-colour operators: vector
and axial bilinears of taste xi_5, (gamma_mu x xi_5)(gamma_mu x xi_5) and
(gamma_mu gamma_5 x xi_5)(gamma_mu gamma_5 x xi_5), mu = 1..4.

Spin and taste labels are 4-bit hypercube masks: bit mu set means a factor
gamma_{mu+1}; gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 is mask 15, and
gamma_mu gamma_5 is mask 15 ^ (1 << mu) up to a sign that cancels between
the two bilinears.
"""

import numpy as np

from .gauge import lattice_volume

XI5 = 15


def propagators(dims, seed, n=4):
    """n Gaussian propagators, each (V, 3, 3) complex128 with re, im ~ N(0, 1),
    drawn one after another from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    vol = lattice_volume(dims)
    out = []
    for _ in range(n):
        g = rng.standard_normal((vol, 3, 3, 2))
        out.append(g[..., 0] + 1j * g[..., 1])
    return out


def bk_ops():
    """(S1, F1, S2, F2) masks of the 8 one-colour B_K-basis operators."""
    vp = [(1 << mu, XI5, 1 << mu, XI5) for mu in range(4)]
    ap = [(XI5 ^ (1 << mu), XI5, XI5 ^ (1 << mu), XI5) for mu in range(4)]
    return vp + ap


def unit_links(dims):
    """Links all equal to the identity, shape (V, 4, 3, 3)."""
    vol = lattice_volume(dims)
    u = np.zeros((vol, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1
    return u
