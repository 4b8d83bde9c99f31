"""Pins of the oracle's asqtad fat links (MILC's path set) and Naik links.

* the fat link equals the direct sum over every path of the action --
  one-link, 6 three-link staples, 24 five-link, 48 seven-link, 6 Lepage --
  each multiplied out step by step with numpy from its list of hops; the
  oracle builds the same sum by nesting whole-lattice staples, so a wrong
  nesting, orientation, dagger or coefficient shows up;
* unit thin links give F = (c1 + 6 c3 + 24 c5 + 48 c7 + 6 cL) 1 = 9/8 1 and
  L = -1/24 1;
* gauge covariance under random SU(3);
* the Naik link over c_N is SU(3).
"""

import numpy as np
import pytest

import oracle
import synth

C1, C3, C5, C7, CL, CN = oracle.ASQTAD_COEFFS


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _path_product(u, dims, path):
    """Product of links along `path` (list of (direction, +-1) hops) from
    every site x, as a (V, 3, 3) array."""
    vol = oracle.volume(dims)
    lex = np.arange(vol)
    shape = (dims[3], dims[2], dims[1], dims[0])
    pos = lex.copy()
    prod = np.broadcast_to(np.eye(3, dtype=np.complex128), (vol, 3, 3)).copy()

    def shift(p, d, k):
        return np.roll(np.arange(vol).reshape(shape), -k, axis=3 - d).reshape(vol)[p]

    for d, s in path:
        if s > 0:
            prod = prod @ u[pos, d]
            pos = shift(pos, d, 1)
        else:
            pos = shift(pos, d, -1)
            prod = prod @ _dag(u[pos, d])
    return prod


def _paths(mu):
    others = [d for d in range(4) if d != mu]
    yield C1, [(mu, 1)]
    for nu in others:
        for s in (1, -1):
            inner = [(nu, s), (mu, 1), (nu, -s)]
            yield C3, inner
            yield CL, [(nu, s), (nu, s), (mu, 1), (nu, -s), (nu, -s)]
            for rho in others:
                if rho == nu:
                    continue
                for r in (1, -1):
                    p5 = [(rho, r)] + inner + [(rho, -r)]
                    yield C5, p5
                    for sg in others:
                        if sg in (nu, rho):
                            continue
                        for q in (1, -1):
                            yield C7, [(sg, q)] + p5 + [(sg, -q)]


def test_path_counts():
    counts = {}
    for c, p in _paths(0):
        counts[len(p)] = counts.get(len(p), 0) + 1
    # 1 one-link; 6 three-link; 24 five-link staples + 6 Lepage; 48 seven-link
    assert counts == {1: 1, 3: 6, 5: 30, 7: 48}


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (2, 4, 6, 4)])
def test_fat_link_is_the_sum_over_paths(dims):
    u = synth.thin_links(dims, 0.5, seed=6)
    fat, lng = oracle.asqtad_links(dims, u)
    vol = oracle.volume(dims)
    for mu in range(4):
        want = np.zeros((vol, 3, 3), dtype=np.complex128)
        for c, p in _paths(mu):
            want += c * _path_product(u, dims, p)
        assert np.abs(fat[:, mu] - want).max() < 1e-13
        naik = CN * _path_product(u, dims, [(mu, 1)] * 3)
        assert np.abs(lng[:, mu] - naik).max() < 1e-15


def test_unit_links():
    dims = (4, 2, 4, 6)
    vol = oracle.volume(dims)
    e = np.broadcast_to(np.eye(3, dtype=np.complex128), (vol, 4, 3, 3)).copy()
    fat, lng = oracle.asqtad_links(dims, e)
    assert C1 + 6 * C3 + 24 * C5 + 48 * C7 + 6 * CL == pytest.approx(9.0 / 8.0, abs=1e-15)
    assert np.abs(fat - 9.0 / 8.0 * np.eye(3)).max() < 1e-15
    assert np.abs(lng - CN * np.eye(3)).max() < 1e-16


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    u = synth.thin_links(dims, 0.8, seed=3)
    g = synth.random_su3(oracle.volume(dims), 2.0, np.random.default_rng(12))
    fat, lng = oracle.asqtad_links(dims, u)
    fg, lg = oracle.asqtad_links(dims, synth.gauge_transform_links(u, g, dims))
    assert np.abs(fg - synth.gauge_transform_links(fat, g, dims)).max() < 1e-13
    assert np.abs(lg - synth.gauge_transform_links(lng, g, dims, hop=3)).max() < 1e-13


def test_naik_is_scaled_su3():
    dims = (4, 4, 2, 4)
    u = synth.thin_links(dims, 0.3, seed=1)
    _, lng = oracle.asqtad_links(dims, u)
    v = lng / CN
    assert np.abs(v @ _dag(v) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(v) - 1).max() < 1e-14
