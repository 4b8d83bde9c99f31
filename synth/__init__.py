"""Seeded synthetic inputs for the asqtad even-odd CG.

This package draws the random inputs that the CUDA library and the CPU oracle
both consume: near-identity SU(3) thin links U = exp(i*eps*H), the synthetic
fat/long link recipe applied to them, Gaussian colour-vector sources and random
gauge transformations.  It holds none of the solver's arithmetic (no Dslash,
no CG); the fat/long recipe is the input recipe of the benchmark workloads, not
the full MILC asqtad path set.

Host layouts (shared by every consumer):

* links: ``[site_lex][mu][row][col]`` complex128, i.e. a numpy array of shape
  ``(V, 4, 3, 3)`` with ``site_lex = x + Lx*(y + Ly*(z + Lz*t))`` and
  ``mu = 0..3`` for ``x, y, z, t``;
* parity-half colour vectors: ``[i][colour]`` complex128, shape ``(V/2, 3)``,
  where ``i = site_lex // 2`` ranks the sites of one parity in lexicographic
  order (valid because ``Lx`` is even).
"""

from .gauge import (  # noqa: F401
    C1, C3, FAT_STAPLE_WEIGHT, gell_mann, random_su3, thin_links, fat_long_links,
    gauge_field, gauge_transform_links, shift_field, lattice_volume,
)
from .fields import gaussian_source, gaussian_sources, parity_sites  # noqa: F401
from . import npr  # noqa: F401
