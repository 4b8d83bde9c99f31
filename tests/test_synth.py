"""Pins of the synthetic input generator (thin links and the fat/long recipe)."""
import numpy as np
import pytest

import synth
from synth.gauge import C1, C3

DIMS = (4, 4, 4, 4)


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


@pytest.mark.parametrize('eps', [0.25, 0.3, 2.0])
def test_thin_links_are_su3(eps):
    u = synth.thin_links(DIMS, eps, seed=3)
    eye = np.eye(3)
    assert np.abs(u @ _dag(u) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14


def test_thin_links_seeded_and_near_identity():
    a = synth.thin_links(DIMS, 0.25, seed=0)
    b = synth.thin_links(DIMS, 0.25, seed=0)
    c = synth.thin_links(DIMS, 0.25, seed=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # exp(i eps H) with eps -> 0 tends to the identity
    small = synth.thin_links(DIMS, 1e-6, seed=0)
    assert np.abs(small - np.eye(3)).max() < 1e-5
    # the generator is exp(i eps H) with H Hermitian traceless:
    # log(U)/(i eps) recovered from U for small eps is Hermitian traceless
    h = (small - np.eye(3)) / (1j * 1e-6)
    assert np.abs(h - _dag(h)).max() < 1e-4
    assert np.abs(np.trace(h, axis1=-2, axis2=-1)).max() < 1e-4


def test_unit_links_give_coefficient_links():
    vol = synth.lattice_volume(DIMS)
    u = np.broadcast_to(np.eye(3, dtype=np.complex128), (vol, 4, 3, 3)).copy()
    fat, lng = synth.fat_long_links(u, DIMS)
    assert np.abs(fat - C1 * np.eye(3)).max() < 1e-15
    assert np.abs(lng - C3 * np.eye(3)).max() < 1e-15


def test_abelian_field_closed_form():
    """U_mu(x) = exp(i theta_mu(x)) * 1: staples reduce to phase sums."""
    dims = (4, 6, 2, 4)
    lx, ly, lz, lt = dims
    vol = synth.lattice_volume(dims)
    rng = np.random.default_rng(5)
    theta = rng.uniform(-np.pi, np.pi, size=(lt, lz, ly, lx, 4))
    u = (np.exp(1j * theta).reshape(vol, 4)[:, :, None, None] * np.eye(3))
    fat, lng = synth.fat_long_links(u, dims)

    def th(mu, shifts):
        # theta_mu at x + sum(shifts), shifts given as {direction: steps}
        a = theta[..., mu]
        for d, k in shifts.items():
            a = np.roll(a, -k, axis=3 - d)
        return a

    for mu in range(4):
        acc = np.exp(1j * th(mu, {}))
        for nu in range(4):
            if nu == mu:
                continue
            acc = acc + 0.1 * np.exp(1j * (th(nu, {}) + th(mu, {nu: 1}) - th(nu, {mu: 1})))
            acc = acc + 0.1 * np.exp(1j * (-th(nu, {nu: -1}) + th(mu, {nu: -1})
                                           + th(nu, {nu: -1, mu: 1})))
        want_f = (C1 * acc / 1.6).reshape(vol)
        want_l = (C3 * np.exp(1j * (th(mu, {}) + th(mu, {mu: 1}) + th(mu, {mu: 2})))).reshape(vol)
        assert np.abs(fat[:, mu, 0, 0] - want_f).max() < 1e-14
        assert np.abs(lng[:, mu, 2, 2] - want_l).max() < 1e-14
        assert np.abs(fat[:, mu, 0, 1]).max() == 0


def test_fat_norm_bound_and_long_is_scaled_su3():
    fat, lng = synth.gauge_field(DIMS, 0.3, seed=0)
    opnorm = np.linalg.norm(fat, ord=2, axis=(-2, -1))
    assert opnorm.max() <= C1 * (1 + 1e-14)
    v = lng / C3
    assert np.abs(v @ _dag(v) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(v) - 1).max() < 1e-14
    # third row of an SU(3) matrix is the conjugated cross product of the first two
    r3 = np.conj(np.cross(v[..., 0, :], v[..., 1, :]))
    assert np.abs(r3 - v[..., 2, :]).max() < 1e-14


def test_builder_is_gauge_covariant():
    u = synth.thin_links(DIMS, 0.3, seed=0)
    g = synth.random_su3(synth.lattice_volume(DIMS), 2.0, np.random.default_rng(99))
    fat, lng = synth.fat_long_links(u, DIMS)
    fat_g, lng_g = synth.fat_long_links(synth.gauge_transform_links(u, g, DIMS), DIMS)
    assert np.abs(fat_g - synth.gauge_transform_links(fat, g, DIMS)).max() < 1e-13
    assert np.abs(lng_g - synth.gauge_transform_links(lng, g, DIMS, hop=3)).max() < 1e-13


def test_gaussian_source_moments_and_seed():
    a = synth.gaussian_source(20000, 0)
    assert a.shape == (20000, 3) and a.dtype == np.complex128
    assert np.array_equal(a, synth.gaussian_source(20000, 0))
    assert abs(a.real.std() - 1) < 0.02 and abs(a.imag.std() - 1) < 0.02
    assert abs(a.mean()) < 0.02
