"""Serving loop (continuous batching) through the C ABI.

Requests on several gauge fields run concurrently; every result passes the
oracle's FP64 residual check; a request gives the same solution alone and in
a busy mix (admissions happen at checkpoint-aligned block boundaries, so the
arithmetic of a system does not depend on its neighbours -- compared within
tol and bit for bit); timeouts, cancellation, bad input and admission under a
tight HBM budget behave as documented.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import gauge

pytestmark = pytest.mark.gpu

FIELDS = [((4, 4, 4, 4), 1), ((8, 8, 4, 8), 2), ((4, 6, 8, 10), 3)]


@pytest.fixture(scope='module')
def served():
    import torch
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1411_2223_gb300 import sq as sqm
    ctx = sqm.Context(0)
    ctx.serve_configure(slots_per_batch=4, block_iters=8)
    gids = {}
    for dims, seed in FIELDS:
        fat, lng = gauge(dims, 0.25, seed)
        gids[dims] = (ctx.gauge_load(dims, fat, lng), fat, lng)
    yield ctx, gids
    ctx.close()


def _req(dims, k):
    vh = oracle.volume(dims) // 2
    rng = np.random.default_rng(100 + k)
    mass = rng.uniform(0.02, 0.1)
    tol = [1e-6, 1e-8][k % 2]
    return synth.gaussian_source(vh, 1000 + k), mass, tol


def test_mixed_stream_matches_oracle(served):
    ctx, gids = served
    tickets = []
    for k in range(18):
        dims = FIELDS[k % 3][0]
        b, m, tol = _req(dims, k)
        tickets.append((ctx.serve_submit(gids[dims][0], b, m, tol), dims, b, m, tol))
    for t, dims, b, m, tol in tickets:
        status, x, st = ctx.serve_poll(t, vh=oracle.volume(dims) // 2, timeout_us=-1)
        assert status == 0 and st['status'] == 0
        _, fat, lng = gids[dims]
        assert oracle.true_residual(dims, fat, lng, m, b, x) <= tol
        assert abs(st['true_residual'] - oracle.true_residual(dims, fat, lng, m, b, x)) <= 1e-3 * tol
    s = ctx.serve_stats()
    assert s['completed'] >= 18 and 0 < s['p50_ms'] <= s['p99_ms']


def test_same_result_alone_and_in_mix(served):
    ctx, gids = served
    dims = (8, 8, 4, 8)
    gid, fat, lng = gids[dims]
    vh = oracle.volume(dims) // 2
    probe = [_req(dims, 40 + k) for k in range(3)]
    alone = []
    for b, m, tol in probe:
        t = ctx.serve_submit(gid, b, m, tol)
        status, x, st = ctx.serve_poll(t, vh=vh, timeout_us=-1)
        assert status == 0
        alone.append((x, st))
    # the same requests inside a busy mix on all fields
    tickets = []
    for k in range(12):
        d = FIELDS[k % 3][0]
        b, m, tol = _req(d, 60 + k)
        tickets.append(ctx.serve_submit(gids[d][0], b, m, tol))
        if k % 4 == 1:
            pb, pm, ptol = probe[k // 4]
            tickets.append(('probe', k // 4, ctx.serve_submit(gid, pb, pm, ptol)))
    for t in tickets:
        if isinstance(t, tuple):
            _, j, tk = t
            status, x, st = ctx.serve_poll(tk, vh=vh, timeout_us=-1)
            assert status == 0
            b, m, tol = probe[j]
            xa, sa = alone[j]
            assert st['iterations'] == sa['iterations']
            assert np.array_equal(x, xa)
            assert np.linalg.norm(x - xa) <= tol * np.linalg.norm(xa)
            assert oracle.true_residual(dims, fat, lng, m, b, x) <= tol
        else:
            assert ctx.serve_poll(t, timeout_us=-1, want_x=False)[0] == 0


def test_poll_timeout_cancel_and_errors(served):
    from paper_1411_2223_gb300 import sq as sqm
    ctx, gids = served
    dims = (4, 6, 8, 10)
    gid = gids[dims][0]
    vh = oracle.volume(dims) // 2
    b = synth.gaussian_source(vh, 7)
    t = ctx.serve_submit(gid, b, 0.005, 1e-10)
    status, _, _ = ctx.serve_poll(t, vh=vh, timeout_us=0)
    assert status in (sqm.PENDING, 0)
    status, x, st = ctx.serve_poll(t, vh=vh, timeout_us=-1)
    assert status == 0
    assert ctx.serve_poll(t, timeout_us=0)[0] == sqm.ERR_NOTFOUND  # released
    t2 = ctx.serve_submit(gid, b, 0.005, 1e-10)
    assert ctx.serve_cancel(t2) == 0
    assert ctx.serve_poll(t2, timeout_us=0)[0] == sqm.ERR_NOTFOUND
    assert ctx.serve_cancel(t2) == sqm.ERR_NOTFOUND
    bad = b.copy()
    bad[0, 0] = np.nan
    with pytest.raises(sqm.SqError) as e:
        ctx.serve_submit(gid, bad, 0.05, 1e-8)
    assert e.value.status == sqm.ERR_NONFINITE
    with pytest.raises(sqm.SqError) as e:
        ctx.serve_submit(gid, b, -0.05, 1e-8)
    assert e.value.status == sqm.ERR_ARG
    with pytest.raises(sqm.SqError) as e:
        ctx.serve_submit(gid + 99, b, 0.05, 1e-8)
    assert e.value.status == sqm.ERR_NOTFOUND
    with pytest.raises(sqm.SqError) as e:
        ctx.serve_configure(2, 8)  # batches exist already
    assert e.value.status == sqm.ERR_BUSY


def test_admission_under_tight_hbm_budget():
    """Budget for the gauge fields plus one batch workspace only: requests on
    the second field wait until the first field's batch is idle and
    released, and every request still completes."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1411_2223_gb300 import sq as sqm
    dims_a, dims_b = (8, 8, 8, 8), (8, 8, 8, 16)
    fa, la = gauge(dims_a, 0.25, 1)
    fb, lb = gauge(dims_b, 0.25, 2)
    ba = synth.gaussian_source(oracle.volume(dims_a) // 2, 500)
    bb = synth.gaussian_source(oracle.volume(dims_b) // 2, 501)
    # measure the footprints with an ample budget
    with sqm.Context(0) as ctx:
        ctx.serve_configure(slots_per_batch=2, block_iters=8)
        ga, gb = ctx.gauge_load(dims_a, fa, la), ctx.gauge_load(dims_b, fb, lb)
        base = ctx.serve_stats()['hbm_in_use']
        ctx.serve_poll(ctx.serve_submit(gb, bb, 0.05, 1e-8), timeout_us=-1, want_x=False)
        with_b = ctx.serve_stats()['hbm_in_use']
        ctx.serve_poll(ctx.serve_submit(ga, ba, 0.05, 1e-8), timeout_us=-1, want_x=False)
        with_ab = ctx.serve_stats()['hbm_in_use']
    batch_b, batch_a = with_b - base, with_ab - with_b
    assert batch_a > 0 and batch_b > 0
    budget = base + max(batch_a, batch_b) + min(batch_a, batch_b) // 2  # one batch at a time
    with sqm.Context(0, hbm_budget=budget) as ctx:
        ctx.serve_configure(slots_per_batch=2, block_iters=8)
        ga, gb = ctx.gauge_load(dims_a, fa, la), ctx.gauge_load(dims_b, fb, lb)
        work = []
        for k in range(6):
            dims, gid, fat, lng = (dims_a, ga, fa, la) if k % 2 == 0 else (dims_b, gb, fb, lb)
            b = synth.gaussian_source(oracle.volume(dims) // 2, 500 + k)
            work.append((ctx.serve_submit(gid, b, 0.05, 1e-8), dims, fat, lng, b))
        for t, dims, fat, lng, b in work:
            status, x, st = ctx.serve_poll(t, vh=oracle.volume(dims) // 2, timeout_us=-1)
            assert status == 0
            assert oracle.true_residual(dims, fat, lng, 0.05, b, x) <= 1e-8
        s = ctx.serve_stats()
        assert s['hbm_in_use'] <= s['hbm_budget'] == budget


def test_full_size_served_requests_match_oracle():
    """The serving workload's own fields at full size (16^3 x 32 and
    20^3 x 64, seeds 2 and 3, eps 0.25): served requests at both
    tolerances, in one mixed stream with a small field beside them, pass the
    oracle's FP64 residual check and agree with the library's own reported
    residual -- the same check as the small lattices, at the volumes the
    benchmark serves."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_1411_2223_gb300 import sq as sqm
    fields = [((16, 16, 16, 32), 2), ((20, 20, 20, 64), 3), ((8, 8, 8, 8), 1)]
    flags = sqm.GAUGE_NO_I16 | sqm.GAUGE_NO_LONG12
    with sqm.Context(0) as ctx:
        ctx.serve_configure(slots_per_batch=8, block_iters=8)
        loaded = []
        for dims, seed in fields:
            fat, lng = synth.gauge_field(dims, 0.25, seed)
            loaded.append((dims, ctx.gauge_load(dims, fat, lng, flags=flags), fat, lng))
        reqs = []
        for k in range(9):
            dims, gid, fat, lng = loaded[k % 3]
            vh = oracle.volume(dims) // 2
            b = synth.gaussian_source(vh, 10000 * (k % 3) + k)
            m = 0.005 + 0.005 * k
            tol = (1e-6, 1e-8)[k % 2]
            reqs.append((ctx.serve_submit(gid, b, m, tol), dims, fat, lng, b, m, tol))
        for t, dims, fat, lng, b, m, tol in reqs:
            status, x, st = ctx.serve_poll(t, vh=oracle.volume(dims) // 2, timeout_us=-1)
            assert status == 0 and st['status'] == 0, (dims, st)
            r = oracle.true_residual(dims, fat, lng, m, b, x)
            assert r <= tol, (dims, m, tol, r)
            assert abs(st['true_residual'] - r) <= 1e-3 * tol
