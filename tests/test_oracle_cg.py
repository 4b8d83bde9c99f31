"""Pins of the oracle's CG, true residual and multi-shift CG.

* free field: a source made of a few even-site plane waves is solved by
  x = sum_k b_k / (m^2 + S(p_k)) (each projected plane wave is an eigenvector
  of A), and CG must terminate after at most as many iterations as there are
  distinct eigenvalues in the source;
* 4^4 random links: the solution equals numpy.linalg.solve on the dense A
  (built column by column from the oracle's Dslash, not from its mdagm);
* multi-shift: every shift equals the dense solve at its own mass.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.gauge import C1, C3


def _s_of(p):
    return sum((C1 * np.sin(q) + C3 * np.sin(3 * q)) ** 2 for q in p)


def _plane_wave_even(dims, n, colour):
    lex = oracle.half_sites(dims, 0)
    lx, ly, lz, lt = dims
    c = np.stack([lex % lx, (lex // lx) % ly, (lex // (lx * ly)) % lz, lex // (lx * ly * lz)], 1)
    p = np.array([2 * np.pi * n[mu] / dims[mu] for mu in range(4)])
    return np.exp(1j * c @ p)[:, None] * np.asarray(colour)[None, :], _s_of(p)


def _unit_links(dims):
    vol = oracle.volume(dims)
    return synth.fat_long_links(np.broadcast_to(np.eye(3, dtype=np.complex128),
                                                (vol, 4, 3, 3)).copy(), dims)


def _dense_a(dims, fat, lng, mass):
    vol = oracle.volume(dims)
    n = 3 * vol
    d = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros((vol, 3), dtype=np.complex128)
    for k in range(n):
        e.reshape(-1)[k] = 1
        d[:, k] = oracle.dslash(dims, fat, lng, e).reshape(-1)
        e.reshape(-1)[k] = 0
    ev = np.concatenate([3 * s + np.arange(3) for s in oracle.half_sites(dims, 0)])
    od = np.concatenate([3 * s + np.arange(3) for s in oracle.half_sites(dims, 1)])
    return mass * mass * np.eye(len(ev)) - d[np.ix_(ev, od)] @ d[np.ix_(od, ev)]


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (8, 4, 4, 8)])
def test_free_field_plane_waves(dims):
    fat, lng = _unit_links(dims)
    mass = 0.05
    rng = np.random.default_rng(0)
    modes = [(1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 1, 1), (0, 0, 0, 1), (1, 0, 1, 3)]
    b = np.zeros((oracle.volume(dims) // 2, 3), dtype=np.complex128)
    x_exact = np.zeros_like(b)
    svals = set()
    for n in modes:
        col = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        pw, s = _plane_wave_even(dims, n, col)
        # each projected plane wave is an eigenvector: A pw = (m^2 + S) pw
        apw = oracle.mdagm(dims, fat, lng, mass, pw)
        assert np.linalg.norm(apw - (mass ** 2 + s) * pw) <= 1e-13 * np.linalg.norm(apw)
        b += pw
        x_exact += pw / (mass ** 2 + s)
        svals.add(round(s, 12))
    x, it, tr = oracle.cg(dims, fat, lng, mass, b, 1e-12)
    assert 0 < it <= len(svals) + 1
    assert tr <= 1e-12
    assert np.linalg.norm(x - x_exact) <= 1e-10 * np.linalg.norm(x_exact)


def test_cg_matches_dense_solve_4444():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    mass = 0.05
    b = synth.gaussian_source(oracle.volume(dims) // 2, 0)
    a = _dense_a(dims, fat, lng, mass)
    x_np = np.linalg.solve(a, b.reshape(-1)).reshape(b.shape)
    x, it, tr = oracle.cg(dims, fat, lng, mass, b, 1e-10)
    assert it > 0 and tr <= 1e-10
    # oracle's own true residual agrees with the dense residual
    dense_res = np.linalg.norm(b.reshape(-1) - a @ x.reshape(-1)) / np.linalg.norm(b)
    assert abs(dense_res - tr) <= 1e-13
    # |x - x*| <= |r| / lambda_min <= |r| / m^2
    assert np.linalg.norm(x - x_np) <= 1.01 * tr * np.linalg.norm(b) / mass ** 2
    x2, it2, tr2 = oracle.cg(dims, fat, lng, mass, b, 1e-12, max_iter=2000)
    assert it2 > 0 and tr2 <= 1e-12
    assert np.linalg.norm(x2 - x_np) <= 1e-9 * np.linalg.norm(x_np)


def test_cg_zero_source_and_max_iter():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    b = np.zeros((oracle.volume(dims) // 2, 3), dtype=np.complex128)
    x, it, tr = oracle.cg(dims, fat, lng, 0.05, b, 1e-10)
    assert it == 0 and np.all(x == 0)
    b = synth.gaussian_source(oracle.volume(dims) // 2, 0)
    x, it, tr = oracle.cg(dims, fat, lng, 0.05, b, 1e-10, max_iter=3)
    assert it == -1 and 0 < tr < 1


def test_multishift_matches_dense_solves():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    masses = 0.05 * 4.0 ** (np.arange(5) / 4.0)
    masses = masses[[2, 0, 4, 1, 3]]           # base (smallest) not first
    b = synth.gaussian_source(oracle.volume(dims) // 2, 1)
    xs, it, tr = oracle.cg_multishift(dims, fat, lng, masses, b, 1e-11)
    assert it > 0
    for i, m in enumerate(masses):
        a = _dense_a(dims, fat, lng, m)
        x_np = np.linalg.solve(a, b.reshape(-1))
        assert tr[i] <= 2e-11
        assert np.linalg.norm(xs[i].reshape(-1) - x_np) <= 1e-8 * np.linalg.norm(x_np)
    # the smallest mass needs as many iterations as the plain CG
    _, it_cg, _ = oracle.cg(dims, fat, lng, masses.min(), b, 1e-11)
    assert abs(it - it_cg) <= 2
