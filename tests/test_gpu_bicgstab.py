"""BiCGstab on the whole-lattice matrix M = m + D (FP64, GPU) vs the FP64
oracle.

Acceptance as for the whole-lattice CG solve: the oracle's own residual
|b - M x| / |b| of the GPU solution is <= tol, and against the oracle's
BiCGstab solution x_ref, |x - x_ref| <= (|b - M x| + |b - M x_ref|) / m
(M^dag M = m^2 - D^2 >= m^2).  The iterates of two BiCGstab runs in
different summation orders drift apart, so iteration counts are compared
loosely.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import gauge

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


@pytest.mark.parametrize('dims,mass', [((4, 4, 4, 4), 0.05), ((4, 6, 8, 10), 0.1),
                                       ((6, 4, 2, 8), 0.2)])
def test_bicgstab_matches_oracle(sq, dims, mass):
    fat, lng = gauge(dims, 0.3, 0)
    b = _src(dims, 2)
    tol = 1e-10
    gid = sq.gauge_load(dims, fat, lng)
    try:
        x, st = sq.bicgstab_solve_full(gid, b, mass, tol)
        assert st['status'] == 0 and st['iterations'] > 0
        x_ref, it_ref, _ = oracle.bicgstab_full(dims, fat, lng, mass, b, tol)
        r = _check(dims, fat, lng, mass, b, x, tol, x_ref)
        assert abs(st['true_residual'] - r) <= 1e-3 * r
        assert st['iterations'] <= 2 * it_ref + 20
    finally:
        sq.gauge_free(gid)


def test_bicgstab_special_cases(sq):
    import torch
    dims = (4, 4, 8, 4)
    fat, lng = gauge(dims, 0.25, 0)
    mass, tol = 0.1, 1e-9
    gid = sq.gauge_load(dims, fat, lng)
    try:
        z = np.zeros((oracle.volume(dims), 3), dtype=np.complex128)
        x, st = sq.bicgstab_solve_full(gid, z, mass, tol)
        assert st['status'] == 0 and st['iterations'] == 0 and not np.any(x)
        b = _src(dims, 5)
        xh, sh = sq.bicgstab_solve_full(gid, b, mass, tol)
        _check(dims, fat, lng, mass, b, xh, tol)
        # device and host pointers give the same bits
        xd, sd = sq.bicgstab_solve_full(gid, torch.from_numpy(b).cuda(), mass, tol)
        assert np.array_equal(xd.cpu().numpy(), xh) and sd['iterations'] == sh['iterations']
        # a solution as initial guess needs no iteration
        xg, sg = sq.bicgstab_solve_full(gid, b, mass, tol, x0=xh)
        assert sg['iterations'] == 0 and sg['status'] == 0
        # max_iter: not converged, x and stats still written
        xm, sm = sq.bicgstab_solve_full(gid, b, mass, 1e-14, max_iter=3, check=False)
        assert sm['status'] == 2 and sm['iterations'] == 3
        # (BiCGstab residuals need not fall monotonically: only its value)
        rm = oracle.full_residual(dims, fat, lng, mass, b, xm)
        assert abs(sm['true_residual'] - rm) <= 1e-9 * rm
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('dims,mass', [((4, 4, 4, 4), 0.05), ((4, 6, 8, 10), 0.1)])
def test_bicgstab_mixed_precision_matches_oracle(sq, dims, mass):
    """FP32 vectors and Dslash with FP64 reliable updates: the same acceptance
    against the oracle's FP64 BiCGstab solution."""
    fat, lng = gauge(dims, 0.3, 0)
    b = _src(dims, 3)
    tol = 1e-10
    gid = sq.gauge_load(dims, fat, lng)
    try:
        x, st = sq.bicgstab_solve_full(gid, b, mass, tol, precision='f32')
        assert st['status'] == 0 and st['reliable_updates'] >= 2
        x_ref, _, _ = oracle.bicgstab_full(dims, fat, lng, mass, b, tol)
        r = _check(dims, fat, lng, mass, b, x, tol, x_ref)
        assert abs(st['true_residual'] - r) <= 1e-3 * r
    finally:
        sq.gauge_free(gid)


def test_bicgstab_full_size_20x64(sq):
    """The benchmark lattice 20^3 x 64 (eps 0.25), am 0.05, tol 1e-8."""
    from paper_1411_2223_gb300 import sq as sqm
    dims = (20, 20, 20, 64)
    fat, lng = gauge(dims, 0.25, 0)
    b = _src(dims, 0)
    gid = sq.gauge_load(dims, fat, lng, flags=sqm.GAUGE_NO_I16 | sqm.GAUGE_NO_LONG12)
    try:
        for prec in ('f64', 'f32'):
            x, st = sq.bicgstab_solve_full(gid, b, 0.05, 1e-8, precision=prec)
            assert st['status'] == 0
            r = _check(dims, fat, lng, 0.05, b, x, 1e-8)
            assert abs(st['true_residual'] - r) <= 1e-4 * r
    finally:
        sq.gauge_free(gid)
