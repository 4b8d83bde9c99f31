"""Whole-lattice solve (m + D) x = b and the unpreconditioned operator on the
GPU vs the FP64 oracle.

A full solve passes when the oracle's own FP64 residual |b - M x| / |b| of
the GPU solution is <= tol and, against the oracle's solution x_ref,
|x - x_ref| <= (|b - M x| + |b - M x_ref|) / m, which holds because
M^dag M = m^2 - D^2 >= m^2.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import gauge, rel, to_dev

pytestmark = pytest.mark.gpu


def _src(dims, seed):
    r = np.random.default_rng(seed)
    v = oracle.volume(dims)
    return r.standard_normal((v, 3)) + 1j * r.standard_normal((v, 3))


def _check(dims, fat, lng, mass, b, x, tol, x_ref=None):
    r = oracle.full_residual(dims, fat, lng, mass, b, x)
    assert r <= tol, r
    if x_ref is not None:
        bn = np.linalg.norm(b)
        r_ref = oracle.full_residual(dims, fat, lng, mass, b, x_ref)
        assert np.linalg.norm(x - x_ref) <= (r + r_ref) * bn / mass * (1 + 1e-9)
    return r


@pytest.mark.parametrize('dims', [(4, 4, 4, 4), (4, 6, 8, 10)])
def test_dirac_apply_matches_oracle(sq, dims):
    import torch
    fat, lng = gauge(dims, 0.25, 0)
    v = _src(dims, 1)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        out = torch.zeros((oracle.volume(dims), 3), dtype=torch.complex128, device='cuda')
        sq.dirac_apply(gid, 0.07, to_dev(v), out)
        got = out.cpu().numpy()
        want = oracle.dirac(dims, fat, lng, 0.07, v)
        assert rel(got, want) <= 1e-13
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec,recon', [('f64', 18), ('f32', 18), ('f32', 12), ('i16', 12)])
def test_full_solve_matches_oracle_4444(sq, prec, recon):
    dims = (4, 4, 4, 4)
    fat, lng = gauge(dims, 0.3, 0)
    b = _src(dims, 2)
    mass, tol = 0.05, 1e-9
    gid = sq.gauge_load(dims, fat, lng)
    try:
        x, st = sq.cg_solve_full(gid, b, mass, tol, precision=prec, long_recon=recon)
        assert st['status'] == 0
        x_ref, _ = oracle.solve_full(dims, fat, lng, mass, b, 1e-13)
        r = _check(dims, fat, lng, mass, b, x, tol, x_ref)
        assert abs(st['true_residual'] - r) <= 1e-6 * r + 1e-15
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec', ['f32', 'i16', 'f64'])
def test_full_solve_ragged_lattice(sq, prec):
    dims = (4, 6, 8, 10)
    fat, lng = gauge(dims, 0.25, 0)
    b = _src(dims, 3)
    mass, tol = 0.03, 1e-8
    gid = sq.gauge_load(dims, fat, lng)
    try:
        x, st = sq.cg_solve_full(gid, b, mass, tol, precision=prec)
        assert st['status'] == 0 and st['iterations'] > 0
        _check(dims, fat, lng, mass, b, x, tol)
    finally:
        sq.gauge_free(gid)


def test_full_solve_special_sources_and_pointers(sq):
    import torch
    dims = (4, 4, 8, 4)
    fat, lng = gauge(dims, 0.25, 0)
    mass, tol = 0.1, 1e-9
    gid = sq.gauge_load(dims, fat, lng)
    try:
        z = np.zeros((oracle.volume(dims), 3), dtype=np.complex128)
        x, st = sq.cg_solve_full(gid, z, mass, tol)
        assert st['status'] == 0 and st['iterations'] == 0 and not np.any(x)
        # odd-only source: x_o = b_o / m exactly where D_eo b_o = 0 is not the case
        b_o = oracle.embed_half(dims, 1, oracle.extract_half(dims, 1, _src(dims, 4)))
        x, st = sq.cg_solve_full(gid, b_o, mass, tol)
        _check(dims, fat, lng, mass, b_o, x, tol)
        # device and host pointers give the same bits
        b = _src(dims, 5)
        xh, sh = sq.cg_solve_full(gid, b, mass, tol)
        xd, sd = sq.cg_solve_full(gid, torch.from_numpy(b).cuda(), mass, tol)
        assert np.array_equal(xd.cpu().numpy(), xh)
        # a solution as initial guess needs no further iterations
        xg, sg = sq.cg_solve_full(gid, b, mass, tol, x0=xh)
        assert sg['iterations'] <= 4
        _check(dims, fat, lng, mass, b, xg, tol)
    finally:
        sq.gauge_free(gid)


def test_full_solve_full_size_20x64(sq):
    """The benchmark lattice 20^3 x 64 (eps 0.25, am 0.01) solved on both
    parities to 1e-8, FP32 CG + FP64 reliable updates."""
    from paper_1411_2223_gb300 import sq as sqm
    dims = (20, 20, 20, 64)
    fat, lng = gauge(dims, 0.25, 0)
    b = _src(dims, 0)
    gid = sq.gauge_load(dims, fat, lng, flags=sqm.GAUGE_NO_I16 | sqm.GAUGE_NO_LONG12)
    try:
        x, st = sq.cg_solve_full(gid, b, 0.01, 1e-8)
        assert st['status'] == 0
        r = _check(dims, fat, lng, 0.01, b, x, 1e-8)
        assert abs(st['true_residual'] - r) <= 1e-4 * r
    finally:
        sq.gauge_free(gid)
