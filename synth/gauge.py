"""Synthetic gauge fields: thin SU(3) links and the fat/long input recipe.

The thin link on every (site, direction) is ``U = exp(i*eps*H)`` with
``H = sum_a omega_a * lambda_a / 2`` (Gell-Mann basis, ``omega_a ~ N(0,1)``).
The exponential is taken through the Hermitian eigendecomposition of H, so U
is unitary with unit determinant to rounding.

Fat and long links follow the benchmark workloads' recipe (an input recipe,
smaller than MILC's asqtad path set):

* ``F_mu(x) = c1 * [U_mu(x) + 0.1 * (sum of the 6 staples around (x, mu))] / 1.6``
  with the up staple ``U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag`` and the down
  staple ``U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)`` for the three nu != mu;
* ``L_mu(x) = c3 * U_mu(x) U_mu(x+mu) U_mu(x+2mu)``;
* ``c1 = 9/8`` and ``c3 = -1/24`` (the tree-level one-hop and Naik
  coefficients) are folded into the stored links, so the Dirac operator that
  consumes them carries no coefficients.

Unit thin links therefore give ``F = c1 * 1`` and ``L = c3 * 1`` exactly.
"""

import numpy as np

C1 = 9.0 / 8.0
C3 = -1.0 / 24.0
FAT_STAPLE_WEIGHT = 0.1


def lattice_volume(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


# numpy axis of each lattice direction mu in a (Lt, Lz, Ly, Lx, ...) array
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def gell_mann():
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def random_su3(n, eps, rng):
    """n SU(3) matrices exp(i*eps*H), H = sum_a omega_a lambda_a / 2.

    Draws ``rng.standard_normal((n, 8))`` (8 normals per matrix, in order).
    """
    omega = rng.standard_normal((n, 8))
    h = np.tensordot(omega, gell_mann() * 0.5, axes=([1], [0]))
    w, v = np.linalg.eigh(h)
    phase = np.exp(1j * eps * w)
    return np.einsum('nij,nj,nkj->nik', v, phase, v.conj())


def thin_links(dims, eps, seed):
    """Thin links, shape (V, 4, 3, 3), drawn site_lex ascending, mu inner."""
    rng = np.random.default_rng(seed)
    vol = lattice_volume(dims)
    return random_su3(vol * 4, eps, rng).reshape(vol, 4, 3, 3)


def shift_field(a, dims, mu, d):
    """Field of shape (V, ...) evaluated at x + d*mu_hat (periodic)."""
    sh = _shape(dims)
    b = a.reshape(sh + a.shape[1:])
    return np.roll(b, -d, axis=_AXIS[mu]).reshape(a.shape)


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def fat_long_links(u, dims, c1=C1, c3=C3, w=FAT_STAPLE_WEIGHT):
    """Fat and long links from thin links u (V, 4, 3, 3) by the input recipe."""
    vol = lattice_volume(dims)
    assert u.shape == (vol, 4, 3, 3)
    fat = np.empty_like(u)
    lng = np.empty_like(u)
    norm = 1.0 + 6.0 * w
    for mu in range(4):
        umu = u[:, mu]
        staples = np.zeros_like(umu)
        for nu in range(4):
            if nu == mu:
                continue
            unu = u[:, nu]
            # up: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
            staples += unu @ shift_field(umu, dims, nu, 1) @ _dag(shift_field(unu, dims, mu, 1))
            # down: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu), built at y = x-nu
            down_at_y = _dag(unu) @ umu @ shift_field(unu, dims, mu, 1)
            staples += shift_field(down_at_y, dims, nu, -1)
        fat[:, mu] = c1 * (umu + w * staples) / norm
        lng[:, mu] = c3 * (umu @ shift_field(umu, dims, mu, 1) @ shift_field(umu, dims, mu, 2))
    return fat, lng


def gauge_field(dims, eps, seed):
    """(fat, long) links of the synthetic near-identity gauge field."""
    return fat_long_links(thin_links(dims, eps, seed), dims)


def gauge_transform_links(u, g, dims, hop=1):
    """U'_mu(x) = g(x) U_mu(x) g(x + hop*mu)^dag for every mu.

    ``hop=1`` transforms thin and fat links, ``hop=3`` transforms long links.
    """
    out = np.empty_like(u)
    for mu in range(4):
        out[:, mu] = g @ u[:, mu] @ _dag(shift_field(g, dims, mu, hop))
    return out
