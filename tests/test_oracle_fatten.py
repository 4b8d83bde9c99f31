"""Pins of the oracle's fat/long link construction (the workloads' recipe):

* unit thin links give F = c1 * 1 and L = c3 * 1 exactly;
* abelian thin links U = exp(i theta) * 1 reduce every staple and the Naik
  product to a sum of phases (closed form);
* gauge covariance with random SU(3) g (non-commuting): F[U^g] = g F g(x+mu)^dag
  and L[U^g] = g L g(x+3mu)^dag -- a wrong order, a missing dagger or a wrong
  neighbour breaks it;
* L / c3 is SU(3), and |F|_op <= c1;
* agreement with the input generator's independent numpy construction.
"""
import numpy as np
import pytest

import oracle
import synth

C1, C3 = oracle.C1, oracle.C3


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def test_unit_links():
    dims = (4, 2, 6, 4)
    vol = oracle.volume(dims)
    u = np.broadcast_to(np.eye(3, dtype=np.complex128), (vol, 4, 3, 3)).copy()
    fat, lng = oracle.fat_long(dims, u)
    assert np.abs(fat - C1 * np.eye(3)).max() < 1e-15
    assert np.abs(lng - C3 * np.eye(3)).max() < 1e-15


def test_abelian_closed_form():
    dims = (4, 6, 2, 4)
    lx, ly, lz, lt = dims
    vol = oracle.volume(dims)
    theta = np.random.default_rng(8).uniform(-np.pi, np.pi, size=(lt, lz, ly, lx, 4))
    u = np.exp(1j * theta).reshape(vol, 4)[:, :, None, None] * np.eye(3)
    w = 0.1
    fat, lng = oracle.fat_long(dims, u, w=w)

    def th(mu, shifts):
        a = theta[..., mu]
        for d, k in shifts.items():
            a = np.roll(a, -k, axis=3 - d)
        return a

    for mu in range(4):
        acc = np.exp(1j * th(mu, {}))
        for nu in set(range(4)) - {mu}:
            acc = acc + w * np.exp(1j * (th(nu, {}) + th(mu, {nu: 1}) - th(nu, {mu: 1})))
            acc = acc + w * np.exp(1j * (-th(nu, {nu: -1}) + th(mu, {nu: -1})
                                         + th(nu, {nu: -1, mu: 1})))
        want_f = (C1 * acc / (1 + 6 * w)).reshape(vol)
        want_l = (C3 * np.exp(1j * (th(mu, {}) + th(mu, {mu: 1}) + th(mu, {mu: 2})))).reshape(vol)
        for c in range(3):
            assert np.abs(fat[:, mu, c, c] - want_f).max() < 1e-14
            assert np.abs(lng[:, mu, c, c] - want_l).max() < 1e-14


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (2, 4, 6, 4)])
def test_gauge_covariance(dims):
    u = synth.thin_links(dims, 0.8, seed=3)
    g = synth.random_su3(oracle.volume(dims), 2.0, np.random.default_rng(11))
    fat, lng = oracle.fat_long(dims, u)
    fat_g, lng_g = oracle.fat_long(dims, synth.gauge_transform_links(u, g, dims))
    assert np.abs(fat_g - synth.gauge_transform_links(fat, g, dims)).max() < 1e-13
    assert np.abs(lng_g - synth.gauge_transform_links(lng, g, dims, hop=3)).max() < 1e-13


def test_long_is_scaled_su3_and_fat_bounded():
    dims = (4, 4, 4, 6)
    u = synth.thin_links(dims, 0.3, seed=0)
    fat, lng = oracle.fat_long(dims, u)
    v = lng / C3
    assert np.abs(v @ _dag(v) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(v) - 1).max() < 1e-14
    assert np.linalg.norm(fat, ord=2, axis=(-2, -1)).max() <= C1 * (1 + 1e-14)


def test_matches_input_generator():
    dims = (4, 6, 4, 4)
    u = synth.thin_links(dims, 0.3, seed=4)
    fat, lng = oracle.fat_long(dims, u)
    f2, l2 = synth.fat_long_links(u, dims)
    assert np.abs(fat - f2).max() < 1e-14 and np.abs(lng - l2).max() < 1e-14
