"""Pins of the oracle's asqtad Dslash and normal operator.

* anti-Hermiticity of D (so D_oe = -D_eo^dag) for random links;
* covariance under random SU(3) gauge transformations;
* the free-field closed form: with unit thin links the eigenvalues of D are
  +-i sqrt(S(p)), S(p) = sum_mu (c1 sin p_mu + c3 sin 3p_mu)^2, and those of
  A = m^2 - D_eo D_oe are m^2 + S(p), every value with half its multiplicity
  over the full momentum set (p_mu = 2 pi n / L_mu; antiperiodic time shifts
  p_t by pi / L_t);
* dense 4^4 brute force with random links: D^dag = -D, spectrum in +-i pairs,
  A Hermitian with lambda_min >= m^2, and the oracle's A equal to the block
  product of its own dense D.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from synth.gauge import C1, C3


def _rand_vec(n, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((n, 3)) + 1j * r.standard_normal((n, 3))


def _unit_links(dims):
    vol = oracle.volume(dims)
    return synth.fat_long_links(np.broadcast_to(np.eye(3, dtype=np.complex128),
                                                (vol, 4, 3, 3)).copy(), dims)


def _dense_d(dims, fat, lng, t_sign=1):
    vol = oracle.volume(dims)
    n = vol * 3
    m = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros((vol, 3), dtype=np.complex128)
    for k in range(n):
        e.reshape(-1)[k] = 1
        m[:, k] = oracle.dslash(dims, fat, lng, e, -1, t_sign).reshape(-1)
        e.reshape(-1)[k] = 0
    return m


def _free_s(dims, t_sign=1):
    ks = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
        if t_sign < 0:
            p[3] += np.pi / dims[3]
        ks.append(sum((C1 * np.sin(q) + C3 * np.sin(3 * q)) ** 2 for q in p))
    return np.array(ks)


@pytest.mark.parametrize('dims,t_sign', [((4, 4, 4, 4), 1), ((4, 4, 2, 6), 1),
                                         ((4, 2, 4, 4), -1), ((8, 4, 4, 4), 1)])
def test_anti_hermitian(dims, t_sign):
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    vol = oracle.volume(dims)
    phi, psi = _rand_vec(vol, 1), _rand_vec(vol, 2)
    lhs = np.vdot(phi, oracle.dslash(dims, fat, lng, psi, -1, t_sign))
    rhs = -np.vdot(oracle.dslash(dims, fat, lng, phi, -1, t_sign), psi)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    # the parity blocks: <phi_e, D_eo psi_o> = -<D_oe phi_e, psi_o>
    pe = oracle.extract_half(dims, 0, phi)
    po = oracle.extract_half(dims, 1, psi)
    a = np.vdot(pe, oracle.dslash_half(dims, fat, lng, po, 0, t_sign))
    b = -np.vdot(oracle.dslash_half(dims, fat, lng, pe, 1, t_sign), po)
    assert abs(a - b) <= 1e-14 * abs(a)


@pytest.mark.parametrize('t_sign', [1, -1])
def test_gauge_covariance(t_sign):
    dims = (4, 4, 4, 6)
    vol = oracle.volume(dims)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    g = synth.random_su3(vol, 2.0, np.random.default_rng(99))
    fat_g = synth.gauge_transform_links(fat, g, dims)
    lng_g = synth.gauge_transform_links(lng, g, dims, hop=3)
    psi = _rand_vec(vol, 4)
    lhs = oracle.dslash(dims, fat_g, lng_g, np.einsum('nij,nj->ni', g, psi), -1, t_sign)
    rhs = np.einsum('nij,nj->ni', g, oracle.dslash(dims, fat, lng, psi, -1, t_sign))
    assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(rhs)


@pytest.mark.parametrize('dims,t_sign', [((4, 4, 4, 4), 1), ((4, 6, 2, 4), 1),
                                         ((4, 4, 4, 4), -1)])
def test_free_field_spectrum(dims, t_sign):
    fat, lng = _unit_links(dims)
    d = _dense_d(dims, fat, lng, t_sign)
    s = np.sort(np.repeat(_free_s(dims, t_sign), 3))
    ev = np.linalg.eigvals(d)
    assert np.abs(ev.real).max() < 1e-13
    # D^2 = -S(p) on plane waves: |eigenvalue|^2 are the S(p), times 3 colours
    assert np.abs(np.sort(ev.imag ** 2) - s).max() < 1e-12
    # the spectrum of D comes in +- pairs
    im = np.sort(ev.imag)
    assert np.abs(im + im[::-1]).max() < 1e-12
    # A on the even sites: m^2 + S(p), each value with half its multiplicity
    m = 0.05
    vh = oracle.volume(dims) // 2
    a = np.zeros((3 * vh, 3 * vh), dtype=np.complex128)
    e = np.zeros((vh, 3), dtype=np.complex128)
    for k in range(3 * vh):
        e.reshape(-1)[k] = 1
        a[:, k] = oracle.mdagm(dims, fat, lng, m, e, t_sign).reshape(-1)
        e.reshape(-1)[k] = 0
    lam = np.linalg.eigvalsh(a)
    assert np.abs(lam - (m * m + s[::2])).max() < 1e-12


def test_dense_random_links_4444():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    d = _dense_d(dims, fat, lng)
    assert np.abs(d + d.conj().T).max() < 1e-15
    ev = np.linalg.eigvals(d)
    assert np.abs(ev.real).max() < 1e-13
    im = np.sort(ev.imag)
    assert np.abs(im + im[::-1]).max() < 1e-12
    # A = m^2 - D_eo D_oe from the dense blocks vs the oracle's mdagm
    ev_idx = np.concatenate([3 * s + np.arange(3) for s in oracle.half_sites(dims, 0)])
    od_idx = np.concatenate([3 * s + np.arange(3) for s in oracle.half_sites(dims, 1)])
    d_eo = d[np.ix_(ev_idx, od_idx)]
    d_oe = d[np.ix_(od_idx, ev_idx)]
    m = 0.05
    a_blocks = m * m * np.eye(len(ev_idx)) - d_eo @ d_oe
    p = _rand_vec(len(ev_idx) // 3, 7)
    got = oracle.mdagm(dims, fat, lng, m, p).reshape(-1)
    assert np.linalg.norm(got - a_blocks @ p.reshape(-1)) <= 1e-14 * np.linalg.norm(got)
    assert np.abs(a_blocks - a_blocks.conj().T).max() < 1e-15
    assert np.linalg.eigvalsh(a_blocks).min() >= m * m * (1 - 1e-10)


def test_dslash_site_matches_full():
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_field(dims, 0.3, seed=0)
    psi = _rand_vec(oracle.volume(dims), 9)
    full = oracle.dslash(dims, fat, lng, psi)
    for s in (0, 1, 17, 255):
        assert np.abs(oracle.dslash_site(dims, fat, lng, psi, s) - full[s]).max() == 0
