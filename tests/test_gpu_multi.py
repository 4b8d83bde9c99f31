"""Batched (multi-RHS) and multi-shift solves vs the FP64 oracle.

Every system of a batch, and every shift, passes the same acceptance as a
single solve: the oracle's FP64 residual <= tol, |A (x - x_ref)|/|b| <= 10 tol
and |x - x_ref| <= (|r| + |r_ref|)/m^2 against the oracle's own solution.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import gauge, o9_check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('prec,recon', [('f32', 18), ('f32', 12), ('i16', 12), ('f64', 18)])
@pytest.mark.parametrize('nrhs', [3, 4, 5])
def test_multi_rhs_matches_oracle(sq, prec, recon, nrhs):
    dims = (4, 6, 8, 10)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    srcs = synth.gaussian_sources(vh, range(nrhs))
    masses = np.linspace(0.03, 0.1, nrhs)
    tol = 1e-8
    gid = sq.gauge_load(dims, fat, lng)
    try:
        xs, stats, status = sq.cg_solve_multi(gid, srcs, masses, tol, precision=prec,
                                              long_recon=recon)
        assert status == 0
        for j in range(nrhs):
            assert stats[j]['status'] == 0
            x_ref, it, _ = oracle.cg(dims, fat, lng, masses[j], srcs[j], 1e-12)
            o9_check(dims, fat, lng, masses[j], srcs[j], xs[j], x_ref, tol)
            # the batched system followed its own recursion: same iteration
            # count as solving it alone
            x1, st1 = sq.cg_solve(gid, srcs[j], masses[j], tol, precision=prec, long_recon=recon)
            assert abs(st1['iterations'] - stats[j]['iterations']) <= 4
    finally:
        sq.gauge_free(gid)


def test_multi_rhs_mixed_convergence_and_zero_source(sq):
    """Systems finish at different iterations; a zero source finishes at once."""
    dims = (8, 4, 4, 8)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    srcs = synth.gaussian_sources(vh, [1, 2, 3])
    srcs[1] = 0
    masses = [0.01, 0.05, 0.3]
    gid = sq.gauge_load(dims, fat, lng)
    try:
        xs, stats, status = sq.cg_solve_multi(gid, srcs, masses, 1e-9)
        assert status == 0
        assert stats[1]['iterations'] == 0 and np.all(xs[1] == 0)
        assert stats[2]['iterations'] < stats[0]['iterations']
        for j in (0, 2):
            assert oracle.true_residual(dims, fat, lng, masses[j], srcs[j], xs[j]) <= 1e-9
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('prec', ['f32', 'i16', 'f64'])
def test_multishift_matches_oracle(sq, prec):
    dims = (4, 4, 4, 8)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    b = synth.gaussian_source(vh, 0)
    # 8 masses from 0.005 to 0.1, geometric, smallest not first
    masses = 0.005 * 20.0 ** (np.arange(8) / 7.0)
    masses = masses[[3, 0, 7, 1, 6, 2, 5, 4]]
    tol = 1e-8
    gid = sq.gauge_load(dims, fat, lng)
    try:
        xs, stats, status = sq.cg_solve_multishift(gid, b, masses, tol, precision=prec)
        assert status == 0
        xo, it_o, tr_o = oracle.cg_multishift(dims, fat, lng, masses, b, 1e-12)
        for i, m in enumerate(masses):
            assert stats[i]['status'] == 0
            o9_check(dims, fat, lng, m, b, xs[i], xo[i], tol)
        # the heaviest shift converges in fewer Krylov steps than the lightest
        assert stats[int(np.argmax(masses))]['iterations'] < stats[int(np.argmin(masses))]['iterations']
    finally:
        sq.gauge_free(gid)


def test_multishift_single_mass_equals_cg(sq):
    dims = (8, 4, 4, 4)
    fat, lng = gauge(dims, 0.25, 0)
    b = synth.gaussian_source(oracle.volume(dims) // 2, 3)
    gid = sq.gauge_load(dims, fat, lng)
    try:
        xs, stats, status = sq.cg_solve_multishift(gid, b, [0.05], 1e-9, precision='f64')
        assert status == 0
        assert oracle.true_residual(dims, fat, lng, 0.05, b, xs[0]) <= 1e-9
    finally:
        sq.gauge_free(gid)


def test_multishift_device_pointers(sq):
    import torch
    dims = (4, 4, 8, 8)
    fat, lng = gauge(dims, 0.25, 0)
    b = synth.gaussian_source(oracle.volume(dims) // 2, 5)
    masses = [0.02, 0.04, 0.08]
    gid = sq.gauge_load(dims, fat, lng)
    try:
        xd, sd, _ = sq.cg_solve_multishift(gid, torch.from_numpy(b).cuda(), masses, 1e-8)
        xh, sh, _ = sq.cg_solve_multishift(gid, b, masses, 1e-8)
        assert np.array_equal(xd.cpu().numpy(), xh)
        for i, m in enumerate(masses):
            assert oracle.true_residual(dims, fat, lng, m, b, xh[i]) <= 1e-8
    finally:
        sq.gauge_free(gid)


def test_batched_full_size_24x64(sq):
    """24^3 x 64, eps 0.25, tol 1e-8: 12 sources (seeds 0..11) at am 0.01 in
    one batched solve, and 8 masses am = 0.005 * 20^(i/7) in one multi-shift
    solve -- the batched workload at full size.  The oracle recomputes the FP64
    residual of every multi-shift solution and of four sampled batch members;
    the rest are checked through the library's FP64 residual."""
    from paper_1411_2223_gb300 import sq as sqm
    dims = (24, 24, 24, 64)
    fat, lng = synth.gauge_field(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    srcs = synth.gaussian_sources(vh, range(12))
    tol = 1e-8
    gid = sq.gauge_load(dims, fat, lng, flags=sqm.GAUGE_NO_I16 | sqm.GAUGE_NO_LONG12)
    try:
        xs, stats, status = sq.cg_solve_multi(gid, srcs, [0.01] * 12, tol)
        assert status == 0
        assert all(s['status'] == 0 and s['true_residual'] <= tol for s in stats)
        for j in (0, 5, 7, 11):
            assert oracle.true_residual(dims, fat, lng, 0.01, srcs[j], xs[j]) <= tol
        masses = 0.005 * 20.0 ** (np.arange(8) / 7.0)
        xm, sm, status = sq.cg_solve_multishift(gid, srcs[0], masses, tol)
        assert status == 0
        for i, m in enumerate(masses):
            assert sm[i]['status'] == 0
            assert oracle.true_residual(dims, fat, lng, m, srcs[0], xm[i]) <= tol
    finally:
        sq.gauge_free(gid)


@pytest.mark.parametrize('nr', [2, 4])
@pytest.mark.parametrize('recon', [18, 12])
def test_many_rhs_tiles_match_oracle(tmp_path, monkeypatch, nr, recon):
    """The FP32 Dslash tiles that apply each link to 2 or 4 systems, forced
    through a tuning cache file (SQ_TUNE_CACHE) onto both kernels of the CG
    iteration (the D_oe kernel with the reduction, mode 3, and the D_eo kernel
    with the update, mode 4) and onto the FP64 reliable-update pair (its
    gated kernels, shape key mode 0), solve every system of a 12-system batch
    with masses 0.02-0.2 (reliable updates for different subsets of the
    systems) to the oracle's acceptance, in the iteration counts of the
    one-system tile (the two tiles add the 16 hop products in different
    orders, so they agree to rounding, not bit for bit).  The solve reports
    the tiles it launched."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1411_2223_gb300 import sq as sqm
    dims = (4, 6, 8, 10)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    nrhs = 12
    srcs = synth.gaussian_sources(vh, range(20, 20 + nrhs))
    masses = np.linspace(0.02, 0.2, nrhs)
    tol = 1e-8
    lat = 'x'.join(map(str, dims))
    results = {}
    for tile in (1, nr):
        cache = tmp_path / ('tune_%d.txt' % tile)
        cache.write_text(''.join('dslash_v4:%s:p1:r%d:n%d:m%d 128 %d\n' % (lat, recon, nrhs, m, tile)
                                 for m in (3, 4)) +
                         'dslash_v4:%s:p0:r18:n%d:m0 128 %d\n' % (lat, nrhs, tile))
        monkeypatch.setenv('SQ_TUNE_CACHE', str(cache))
        with sqm.Context(0) as ctx:
            gid = ctx.gauge_load(dims, fat, lng)
            xs, stats, status = ctx.cg_solve_multi(gid, srcs, masses, tol, long_recon=recon)
            assert status == 0
        for s in stats:
            assert (s['oe_rhs_tile'], s['eo_rhs_tile']) == (tile, tile), s
            assert (s['oe_block'], s['eo_block']) == (128, 128), s
        results[tile] = (xs, [s['iterations'] for s in stats])
    xs, its = results[nr]
    assert max(abs(a - b) for a, b in zip(its, results[1][1])) <= 4
    for j in range(nrhs):
        x_ref, _, _ = oracle.cg(dims, fat, lng, masses[j], srcs[j], 1e-12)
        o9_check(dims, fat, lng, masses[j], srcs[j], xs[j], x_ref, tol)


TILES = {'f32': (1, 2, 4), 'f64': (1, 2, 4), 'i16': (1, 2, 4)}


@pytest.mark.parametrize('prec', ['f32', 'f64', 'i16'])
@pytest.mark.parametrize('recon', [18, 12])
def test_batched_dslash_every_tile_matches_oracle(tmp_path, monkeypatch, prec, recon):
    """dslash_apply_multi on 12 right-hand sides with each tile of
    right-hand sides per thread forced through SQ_TUNE_CACHE: every system's
    output matches the oracle's Dslash on the unquantised input, in norm and
    site by site (a 2 x 6 x 4 x 10 lattice: 240 sites per parity, ragged
    against every block, several tiles of the 12 systems and a partial last
    one), and sq_tuned_launch reports the forced shape."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1411_2223_gb300 import sq as sqm
    from gpu_helpers import TOL_DSLASH, rel, site_rel
    dims = (2, 6, 4, 10)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    nrhs = 12
    srcs = synth.gaussian_sources(vh, range(40, 40 + nrhs))
    lat = 'x'.join(map(str, dims))
    want = [[oracle.dslash_half(dims, fat, lng, srcs[j], par) for j in range(nrhs)]
            for par in (0, 1)]
    for tile in TILES[prec]:
        cache = tmp_path / ('tune_%s_%d.txt' % (prec, tile))
        cache.write_text('dslash_v4:%s:p%d:r%d:n%d:m0 128 %d\n'
                         % (lat, sqm.PREC[prec], recon, nrhs, tile))
        monkeypatch.setenv('SQ_TUNE_CACHE', str(cache))
        with sqm.Context(0) as ctx:
            gid = ctx.gauge_load(dims, fat, lng)
            assert ctx.tuned_launch(gid, prec, recon, nrhs, 'plain') == (128, tile)
            nbytes, _ = ctx.spinor_bytes(gid, prec)
            src = torch.zeros(nrhs * nbytes, dtype=torch.uint8, device='cuda')
            dst = torch.zeros_like(src)
            for j in range(nrhs):
                ctx.pack_spinor(gid, prec, torch.from_numpy(srcs[j]).cuda(),
                                src[j * nbytes:(j + 1) * nbytes])
            for par in (0, 1):
                ctx.dslash_apply_multi(gid, par, prec, recon, nrhs, src, dst)
                for j in range(nrhs):
                    canon = torch.zeros((vh, 3), dtype=torch.complex128, device='cuda')
                    ctx.unpack_spinor(gid, prec, dst[j * nbytes:(j + 1) * nbytes], canon)
                    got = canon.cpu().numpy()
                    w = want[par][j]
                    assert rel(got, w) <= TOL_DSLASH[prec], (tile, par, j, rel(got, w))
                    assert site_rel(got, w) <= TOL_DSLASH[prec], (tile, par, j)


def test_batched_entry_points_reject_bad_arguments(sq):
    """dslash_apply_multi, sq_tuned_launch and sq_time_dslash refuse bad
    batch sizes, modes, precisions and unknown gauge ids with the documented
    statuses, and sq_time_dslash times the CG's kernels at a positive
    duration on a real field."""
    import torch
    from paper_1411_2223_gb300 import sq as sqm
    dims = (4, 4, 4, 8)
    fat, lng = gauge(dims, 0.25, 0)
    gid = sq.gauge_load(dims, fat, lng, flags=sqm.GAUGE_NO_I16)
    try:
        nbytes, _ = sq.spinor_bytes(gid, 'f32')
        a = torch.zeros(2 * nbytes, dtype=torch.uint8, device='cuda')
        b = torch.zeros_like(a)
        cases = [
            (lambda: sq.dslash_apply_multi(gid, 0, 'f32', 18, 0, a, b), sqm.ERR_ARG),
            (lambda: sq.dslash_apply_multi(gid, 0, 'f32', 18, 65, a, b), sqm.ERR_ARG),
            (lambda: sq.dslash_apply_multi(gid, 2, 'f32', 18, 2, a, b), sqm.ERR_ARG),
            (lambda: sq.dslash_apply_multi(gid, 0, 'f32', 18, 2, a, a), sqm.ERR_ARG),
            (lambda: sq.dslash_apply_multi(gid + 99, 0, 'f32', 18, 2, a, b), sqm.ERR_NOTFOUND),
            (lambda: sq.dslash_apply_multi(gid, 0, 'i16', 18, 2, a, b), sqm.ERR_UNSUPPORTED),
            (lambda: sq.tuned_launch(gid, 'f32', 18, 4, 2), sqm.ERR_ARG),      # mode 2: FP64 only
            (lambda: sq.tuned_launch(gid, 'f32', 11, 4, 'plain'), sqm.ERR_ARG),
            (lambda: sq.tuned_launch(gid + 99, 'f32', 18, 4, 'plain'), sqm.ERR_NOTFOUND),
            (lambda: sq.time_dslash(gid, 'f32', 18, 1, 'cg_oe', reps=0), sqm.ERR_ARG),
            (lambda: sq.time_dslash(gid, 'f32', 18, 0, 'cg_oe'), sqm.ERR_ARG),
        ]
        for k, (call, status) in enumerate(cases):
            with pytest.raises(sqm.SqError) as e:
                call()
            assert e.value.status == status, k
        for mode in ('plain', 'cg_oe', 'cg_eo'):
            assert 0.0 < sq.time_dslash(gid, 'f32', 18, 4, mode, reps=3) < 1e5
    finally:
        sq.gauge_free(gid)


def test_64_system_batch_matches_oracle(sq):
    """The largest batch, 64 systems with 64 masses from 0.02 to 0.5 (the
    systems converge, and need their reliable updates, at different
    iterations): the reliable-update kernels' active-tile mask then spans
    both halves of its 64 bits.  Every system meets the oracle's residual."""
    dims = (4, 4, 4, 6)
    fat, lng = gauge(dims, 0.25, 0)
    vh = oracle.volume(dims) // 2
    nrhs = 64
    srcs = synth.gaussian_sources(vh, range(100, 100 + nrhs))
    masses = np.geomspace(0.02, 0.5, nrhs)
    tol = 1e-8
    gid = sq.gauge_load(dims, fat, lng)
    try:
        xs, stats, status = sq.cg_solve_multi(gid, srcs, masses, tol)
        assert status == 0
        its = [s['iterations'] for s in stats]
        assert its[0] > its[-1]
        for j in range(nrhs):
            assert stats[j]['status'] == 0
            assert oracle.true_residual(dims, fat, lng, masses[j], srcs[j], xs[j]) <= tol
    finally:
        sq.gauge_free(gid)
