"""Pins of the oracle's whole-lattice staggered matrix M = m + D and of its
full-lattice solve by even-odd reduction.

* M^dag M = (m - D)(m + D) restricted to the even sites equals the oracle's
  separately written normal operator m^2 - D_eo D_oe (anti-Hermitian D);
* on a 4^4 lattice with random links the even-odd solve agrees with
  numpy.linalg.solve on the dense 768 x 768 M built column by column, and the
  dense solution has a full residual at rounding level;
* with unit links a plane wave is an eigenvector of D, so M x = b has the
  closed-form solution x = b (m - i s) / (m^2 + s^2) on each momentum's
  two-dimensional D-invariant space -- checked through the residual;
* zero and odd-only sources reduce as the algebra says.
"""
import numpy as np
import pytest

import oracle
import synth


def _rand_full(dims, seed):
    r = np.random.default_rng(seed)
    v = oracle.volume(dims)
    return r.standard_normal((v, 3)) + 1j * r.standard_normal((v, 3))


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (4, 6, 2, 4)])
def test_mdagm_is_even_block_of_m_dag_m(dims):
    fat, lng = synth.gauge_field(dims, 0.3, seed=1)
    mass = 0.07
    v = oracle.extract_half(dims, 0, _rand_full(dims, 3))
    w = oracle.dirac(dims, fat, lng, mass, oracle.embed_half(dims, 0, v))
    # (m - D) w = -((-m) + D) w
    y = -oracle.dirac(dims, fat, lng, -mass, w)
    want = oracle.mdagm(dims, fat, lng, mass, v)
    got = oracle.extract_half(dims, 0, y)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
    # and M^dag M has no even -> odd block
    assert np.linalg.norm(oracle.extract_half(dims, 1, y)) <= 1e-13 * np.linalg.norm(want)


def test_solve_full_matches_dense_solve_4444():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    mass = 0.05
    vol = oracle.volume(dims)
    n = 3 * vol
    dense = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros((vol, 3), dtype=np.complex128)
    for k in range(n):
        e.reshape(-1)[k] = 1
        dense[:, k] = oracle.dirac(dims, fat, lng, mass, e).reshape(-1)
        e.reshape(-1)[k] = 0
    b = _rand_full(dims, 5)
    x_dense = np.linalg.solve(dense, b.reshape(-1)).reshape(vol, 3)
    assert oracle.full_residual(dims, fat, lng, mass, b, x_dense) <= 1e-13
    x, it = oracle.solve_full(dims, fat, lng, mass, b, 1e-12)
    assert it > 0
    assert oracle.full_residual(dims, fat, lng, mass, b, x) <= 1e-12
    assert np.linalg.norm(x - x_dense) <= 1e-9 * np.linalg.norm(x_dense)
    # the residual the function reports is |b - M x| for any x
    d = _rand_full(dims, 9) * 1e-3
    want = np.linalg.norm(dense @ d.reshape(-1)) / np.linalg.norm(b)
    assert abs(oracle.full_residual(dims, fat, lng, mass, b, x_dense + d) - want) <= 1e-9 * want


def test_free_field_plane_wave_solution():
    """Unit links: D e^{ipx} c is not a multiple of e^{ipx} (the eta phases
    mix momenta p and p + pi), but M^dag M = m^2 - D^2 is diagonal in p with
    eigenvalue m^2 + S(p); so x = (m - D) b / (m^2 + S(p)) solves M x = b for
    a plane-wave b."""
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
    b = phase[:, None] * np.array([1.0, -0.5j, 0.25])[None, :]
    s = sum((C1 * np.sin(q) + C3 * np.sin(3 * q)) ** 2 for q in p)
    mass = 0.1
    x = (mass * b - oracle.dslash(dims, fat, lng, b)) / (mass ** 2 + s)
    assert oracle.full_residual(dims, fat, lng, mass, b, x) <= 1e-14
    xs, _ = oracle.solve_full(dims, fat, lng, mass, b, 1e-13)
    assert np.linalg.norm(xs - x) <= 1e-11 * np.linalg.norm(x)


def test_zero_and_odd_only_sources():
    dims = (4, 4, 2, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=2)
    mass = 0.2
    z = np.zeros((oracle.volume(dims), 3), dtype=np.complex128)
    x, it = oracle.solve_full(dims, fat, lng, mass, z, 1e-10)
    assert it == 0 and not np.any(x)
    b_o = oracle.embed_half(dims, 1, oracle.extract_half(dims, 1, _rand_full(dims, 4)))
    x, _ = oracle.solve_full(dims, fat, lng, mass, b_o, 1e-12)
    assert oracle.full_residual(dims, fat, lng, mass, b_o, x) <= 1e-12
