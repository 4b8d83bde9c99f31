"""Pins of the oracle's lattice layer: coordinates, neighbours, phases.

Checked against brute force over explicit coordinates and against the
staggered-phase anticommutation identity, which any correct choice of
Kawamoto-Smit phases satisfies.
"""
import itertools

import numpy as np
import pytest

import oracle

DIMS = [(4, 4, 4, 4), (4, 6, 2, 8), (6, 2, 4, 4)]


def _coords(dims, s):
    lx, ly, lz, lt = dims
    return (s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz))


@pytest.mark.parametrize('dims', DIMS)
def test_neighbors_brute_force(dims):
    lx, ly, lz, lt = dims
    L = dims
    for s in range(oracle.volume(dims)):
        c = _coords(dims, s)
        for mu in range(4):
            for d in (1, -1, 3, -3):
                cc = list(c)
                cc[mu] = (cc[mu] + d) % L[mu]
                want = cc[0] + lx * (cc[1] + ly * (cc[2] + lz * cc[3]))
                got, sign = oracle.neighbor(dims, s, mu, d)
                assert got == want and sign == 1


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (2, 2, 2, 2), (4, 2, 2, 6)])
def test_antiperiodic_sign_counts_wraps(dims):
    lt = dims[3]
    for s in range(oracle.volume(dims)):
        t = _coords(dims, s)[3]
        for d in (1, -1, 3, -3):
            wraps = (t + d) // lt          # python floor division
            _, sign = oracle.neighbor(dims, s, 3, d, t_sign=-1)
            assert sign == (-1 if wraps % 2 else 1)
            for mu in range(3):
                assert oracle.neighbor(dims, s, mu, d, t_sign=-1)[1] == 1


@pytest.mark.parametrize('dims', DIMS)
def test_parity_and_half_index(dims):
    vol = oracle.volume(dims)
    for p in (0, 1):
        lex = oracle.half_sites(dims, p)
        assert len(lex) == vol // 2
        # the half-lattice index of a site is site_lex // 2
        assert np.array_equal(lex // 2, np.arange(vol // 2))
        for s in lex[:: max(1, len(lex) // 50)]:
            assert oracle.parity(dims, s) == p == sum(_coords(dims, s)) % 2


@pytest.mark.parametrize('dims', DIMS)
def test_eta_values_and_anticommutation(dims):
    vol = oracle.volume(dims)
    for s in range(vol):
        x, y, z, t = _coords(dims, s)
        assert oracle.eta(dims, s, 0) == 1
        assert oracle.eta(dims, s, 1) == (-1) ** x
        assert oracle.eta(dims, s, 2) == (-1) ** (x + y)
        assert oracle.eta(dims, s, 3) == (-1) ** (x + y + z)
        # eta_mu(x) eta_nu(x+mu) = - eta_nu(x) eta_mu(x+nu), mu != nu
        for mu, nu in itertools.permutations(range(4), 2):
            xm, _ = oracle.neighbor(dims, s, mu, 1)
            xn, _ = oracle.neighbor(dims, s, nu, 1)
            lhs = oracle.eta(dims, s, mu) * oracle.eta(dims, xm, nu)
            rhs = -oracle.eta(dims, s, nu) * oracle.eta(dims, xn, mu)
            assert lhs == rhs
