"""Pins of the oracle's BiCGstab solve of the whole-lattice staggered matrix
M = m + D (the BiCG-family inverter named in Sec. 3):

* on a 4^4 lattice with random links it agrees with numpy.linalg.solve on
  the dense 768 x 768 M built column by column (within the rigorous bound
  |x - x*| <= |r| / sigma_min(M) = |r| / m, since M^dag M >= m^2);
* with unit links a plane-wave source has the closed-form solution
  x = (m - D) b / (m^2 + S(p)), S(p) = sum_mu (c1 sin p_mu + c3 sin 3 p_mu)^2;
* it reports the residual that the dense operator gives, and a zero source
  needs no iteration.
"""
import numpy as np
import pytest

import oracle
import synth


def _rand_full(dims, seed):
    r = np.random.default_rng(seed)
    v = oracle.volume(dims)
    return r.standard_normal((v, 3)) + 1j * r.standard_normal((v, 3))


def _dense_m(dims, fat, lng, mass):
    vol = oracle.volume(dims)
    n = 3 * vol
    dense = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros((vol, 3), dtype=np.complex128)
    for k in range(n):
        e.reshape(-1)[k] = 1
        dense[:, k] = oracle.dirac(dims, fat, lng, mass, e).reshape(-1)
        e.reshape(-1)[k] = 0
    return dense


@pytest.mark.parametrize('mass,tol', [(0.05, 1e-10), (0.2, 1e-12)])
def test_bicgstab_matches_dense_solve_4444(mass, tol):
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    dense = _dense_m(dims, fat, lng, mass)
    b = _rand_full(dims, 5)
    x_star = np.linalg.solve(dense, b.reshape(-1))
    x, it, res = oracle.bicgstab_full(dims, fat, lng, mass, b, tol)
    assert it > 0 and res <= tol
    r = b.reshape(-1) - dense @ x.reshape(-1)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - res) <= 1e-3 * res + 1e-15
    assert np.linalg.norm(x.reshape(-1) - x_star) <= (np.linalg.norm(r) / mass) * (1 + 1e-6) \
        + 1e-12 * np.linalg.norm(x_star)


def test_bicgstab_free_field_plane_wave():
    from synth.gauge import C1, C3
    dims = (4, 4, 6, 4)
    vol = oracle.volume(dims)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (vol, 4, 3, 3)).copy()
    fat, lng = synth.fat_long_links(eye, dims)
    lex = np.arange(vol)
    coords = [lex % 4, (lex // 4) % 4, (lex // 16) % 6, lex // 96]
    n = (1, 0, 2, 3)
    p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
    phase = np.exp(1j * sum(p[mu] * coords[mu] for mu in range(4)))
    b = phase[:, None] * np.array([0.3 - 0.2j, 1.0, -0.5j])[None, :]
    mass = 0.1
    s = sum((C1 * np.sin(p[mu]) + C3 * np.sin(3 * p[mu])) ** 2 for mu in range(4))
    want = oracle.dirac(dims, fat, lng, -mass, b) * (-1) / (mass ** 2 + s)
    x, it, res = oracle.bicgstab_full(dims, fat, lng, mass, b, 1e-12)
    assert res <= 1e-12
    assert np.linalg.norm(x - want) <= 1e-10 * np.linalg.norm(want)


def test_bicgstab_zero_source():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    x, it, res = oracle.bicgstab_full(dims, fat, lng, 0.1, np.zeros((256, 3), complex), 1e-10)
    assert it == 0 and res == 0.0 and not x.any()
