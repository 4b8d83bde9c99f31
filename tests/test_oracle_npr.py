"""Pins of the oracle's NPR four-fermion operator (Eq. 1).

Spin-taste matrices (computed in the oracle from explicit 4 x 4 Dirac
matrices and traces) against the textbook phases of the staggered hypercube:
* (gamma_mu x 1) is the one-link shift with the staggered phase eta_mu(A),
  the same eta the Dslash uses (taken from the oracle's lattice phase);
* (1 x xi_mu) is the shift with the taste phase zeta_mu(A) =
  (-1)^(sum_{nu > mu} A_nu);
* every (gamma_S x xi_F) is the ordered product of those shifts, and
  (gamma_5 x xi_5) is the parity phase (-1)^|A| -- a dropped dagger, a
  transposed matrix or a wrong sign in the trace fails these.

Averaged links against closed forms: unit links give 1, pure-gauge links
U_mu(x) = g(x) g(x+mu)^dag give g(z_A) g(z_D)^dag on every path, one-link
pairs give the link or its dagger, two-link pairs the mean of the two
plaquette halves, and U_DA = U_AD^dag.

The contraction against:
* gauge invariance on every hypercube (links U -> g U g^dag, propagators
  G -> g G) with non-commuting g;
* fields supported on one corner per flavour, where Eq. 1 reduces to one
  term M1[A][B] M2[C][D] (g1^dag U_AD g4)[a1][a4] (g3^dag U_CB g2)[a3][a2]
  -- a swapped flavour, colour pairing or corner fails it;
* unit links and constant fields, where the sum factorises into the sums of
  the spin-taste matrices times (G1^dag G4) (x) (G3^dag G2).
"""
import itertools

import numpy as np

import oracle
import synth
from synth import npr as snpr


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _bits(a):
    return [(a >> mu) & 1 for mu in range(4)]


def _corner_lex(dims, z, a):
    c = [2 * z[mu] + ((a >> mu) & 1) for mu in range(4)]
    return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))


def _eta_shift(dims, mu):
    """(gamma_mu x 1) from the lattice phase eta_mu at the corners of
    hypercube 0 (a standalone closed form: eta_mu(A) delta_{B, A^mu})."""
    m = np.zeros((16, 16))
    for a in range(16):
        m[a, a ^ (1 << mu)] = oracle.eta(dims, _corner_lex(dims, (0, 0, 0, 0), a), mu)
    return m


def _zeta_shift(mu):
    m = np.zeros((16, 16))
    for a in range(16):
        m[a, a ^ (1 << mu)] = (-1) ** sum(_bits(a)[mu + 1:])
    return m


def _shift_product(dims, s, f):
    m = np.eye(16)
    for mu in range(4):
        if (s >> mu) & 1:
            m = m @ _eta_shift(dims, mu)
    for mu in range(4):
        if (f >> mu) & 1:
            m = m @ _zeta_shift(mu)
    return m


def test_gammas_clifford():
    g = oracle.gammas()
    for mu in range(4):
        assert np.abs(g[mu] - g[mu].conj().T).max() == 0
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.abs(ac - 2 * (mu == nu) * np.eye(4)).max() < 1e-15


def test_spin_taste_eta_zeta_eps():
    dims = (4, 4, 4, 4)
    # the staggered phase of the Dslash: eta_mu(A) = (-1)^(sum_{nu < mu} A_nu)
    for mu in range(4):
        for a in range(16):
            assert _eta_shift(dims, mu)[a, a ^ (1 << mu)] == (-1) ** sum(_bits(a)[:mu])
        assert np.abs(oracle.spin_taste(1 << mu, 0) - _eta_shift(dims, mu)).max() < 1e-15
        assert np.abs(oracle.spin_taste(0, 1 << mu) - _zeta_shift(mu)).max() < 1e-15
    assert np.abs(oracle.spin_taste(0, 0) - np.eye(16)).max() < 1e-15
    eps = np.diag([(-1.0) ** sum(_bits(a)) for a in range(16)])
    assert np.abs(oracle.spin_taste(15, 15) - eps).max() < 1e-15


def test_spin_taste_all_from_shifts():
    dims = (4, 4, 4, 4)
    for s in range(16):
        for f in range(16):
            m = oracle.spin_taste(s, f)
            assert np.abs(m - _shift_product(dims, s, f)).max() < 1e-14, (s, f)
            assert np.abs(m @ m.conj().T - np.eye(16)).max() < 1e-14


def test_avg_link_unit_and_pure_gauge():
    dims = (4, 6, 4, 8)
    vol = oracle.volume(dims)
    u1 = snpr.unit_links(dims)
    g = synth.random_su3(vol, 2.0, np.random.default_rng(99))
    ug = synth.gauge_transform_links(u1, g, dims)
    for z in [(0, 0, 0, 0), (1, 2, 1, 3), (1, 1, 0, 2)]:
        for a in range(16):
            for d in range(16):
                assert np.abs(oracle.npr_avg_link(dims, u1, z, a, d) - np.eye(3)).max() < 1e-15
                want = g[_corner_lex(dims, z, a)] @ _dag(g[_corner_lex(dims, z, d)])
                got = oracle.npr_avg_link(dims, ug, z, a, d)
                assert np.abs(got - want).max() < 1e-13, (z, a, d)


def test_avg_link_short_paths_and_reverse():
    dims = (4, 4, 6, 4)
    u = synth.thin_links(dims, 0.4, 5)
    z = (1, 0, 2, 1)
    site = lambda a: _corner_lex(dims, z, a)
    for a in range(16):
        for mu in range(4):
            d = a ^ (1 << mu)
            got = oracle.npr_avg_link(dims, u, z, a, d)
            want = u[site(a), mu] if not (a >> mu) & 1 else _dag(u[site(d), mu])
            assert np.abs(got - want).max() < 1e-15
    for mu, nu in itertools.combinations(range(4), 2):
        d = (1 << mu) | (1 << nu)
        want = 0.5 * (u[site(0), mu] @ u[site(1 << mu), nu] +
                      u[site(0), nu] @ u[site(1 << nu), mu])
        assert np.abs(oracle.npr_avg_link(dims, u, z, 0, d) - want).max() < 1e-15
    for a in range(16):
        for d in range(16):
            uad = oracle.npr_avg_link(dims, u, z, a, d)
            uda = oracle.npr_avg_link(dims, u, z, d, a)
            assert np.abs(uda - _dag(uad)).max() < 1e-15


def test_four_fermion_gauge_invariance():
    dims = (4, 4, 4, 6)
    vol = oracle.volume(dims)
    u = synth.thin_links(dims, 0.5, 3)
    props = snpr.propagators(dims, 11)
    ops = [snpr.bk_ops()[1], snpr.bk_ops()[6], (3, 5, 12, 9)]
    o = oracle.npr_four_fermion(dims, u, props, ops)
    g = synth.random_su3(vol, 2.0, np.random.default_rng(99))
    ug = synth.gauge_transform_links(u, g, dims)
    pg = [g @ p for p in props]
    og = oracle.npr_four_fermion(dims, ug, pg, ops)
    scale = np.abs(o).max()
    assert scale > 1
    assert np.abs(og - o).max() < 1e-12 * scale


def test_four_fermion_single_corner_fields():
    dims = (4, 4, 4, 4)
    vol = oracle.volume(dims)
    rng = np.random.default_rng(4)
    g = synth.random_su3(vol, 2.0, rng)
    ug = synth.gauge_transform_links(snpr.unit_links(dims), g, dims)
    z0 = (1, 0, 1, 1)
    zi = oracle.hypercube_index(dims, z0)
    op = (1, 3, 12, 9)            # gamma_1 x xi_1 xi_2, gamma_3 gamma_4 x xi_1 xi_4
    m1 = _shift_product(dims, op[0], op[1])
    m2 = _shift_product(dims, op[2], op[3])
    t1, t2 = op[0] ^ op[1], op[2] ^ op[3]
    # M1 is antisymmetric: a corner where swapping A and B flips the sign
    a0 = next(a for a in range(16) if m1[a, a ^ t1] != m1[a ^ t1, a])
    b0 = a0 ^ t1
    c0 = 6
    d0 = c0 ^ t2
    gm = [rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)) for _ in range(4)]
    props = [np.zeros((vol, 3, 3), dtype=np.complex128) for _ in range(4)]
    for f, corner in enumerate((a0, b0, c0, d0)):
        props[f][_corner_lex(dims, z0, corner)] = gm[f]
    o = oracle.npr_four_fermion(dims, ug, props, [op])
    site = lambda a: _corner_lex(dims, z0, a)
    u_ad = g[site(a0)] @ _dag(g[site(d0)])
    u_cb = g[site(c0)] @ _dag(g[site(b0)])
    p14 = _dag(gm[0]) @ u_ad @ gm[3]
    p32 = _dag(gm[2]) @ u_cb @ gm[1]
    want = m1[a0, b0] * m2[c0, d0] * np.einsum('il,kj->ijkl', p14, p32)
    assert np.abs(o[zi, 0] - want).max() < 1e-13 * np.abs(want).max()
    others = np.delete(o[:, 0], zi, axis=0)
    assert np.abs(others).max() == 0
    # corners that the spin-taste matrices do not join give nothing
    props[1][:] = 0
    props[1][site(b0 ^ 1)] = gm[1]
    assert np.abs(oracle.npr_four_fermion(dims, ug, props, [op])).max() == 0


def test_four_fermion_unit_links_constant_fields():
    dims = (4, 4, 6, 4)
    vol = oracle.volume(dims)
    rng = np.random.default_rng(12)
    gm = [rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)) for _ in range(4)]
    props = [np.broadcast_to(m, (vol, 3, 3)).copy() for m in gm]
    ops = snpr.bk_ops()[:2] + [(0, 0, 15, 15), (3, 5, 12, 9)]
    o = oracle.npr_four_fermion(dims, snpr.unit_links(dims), props, ops)
    p14 = _dag(gm[0]) @ gm[3]
    p32 = _dag(gm[2]) @ gm[1]
    outer = np.einsum('il,kj->ijkl', p14, p32)
    for k, op in enumerate(ops):
        s1 = _shift_product(dims, op[0], op[1]).sum()
        s2 = _shift_product(dims, op[2], op[3]).sum()
        want = s1 * s2 * outer
        assert np.abs(o[:, k] - want).max() < 1e-12 * max(1.0, np.abs(outer).max()), op


def test_hypercube_subset_matches_all():
    dims = (4, 4, 4, 4)
    u = synth.thin_links(dims, 0.3, 2)
    props = snpr.propagators(dims, 3)
    ops = snpr.bk_ops()[:3]
    full = oracle.npr_four_fermion(dims, u, props, ops)
    sub = oracle.npr_four_fermion(dims, u, props, ops, hypercubes=[5, 0, 15])
    assert np.array_equal(sub, full[[5, 0, 15]])
