#!/usr/bin/env python
"""Benchmark of the asqtad mixed-precision CG on one GB300 (or N replicas).

Workload (the paper's lattice shape, Sec. 2 / Fig. 1): a 20^3 x 64 synthetic
near-identity gauge field (thin links exp(i 0.25 H), seed 0, fat/long input
recipe), Gaussian source (seed 0), am = 0.01, relative residual 1e-8.

One step = one solve of (m^2 - D_eo D_oe) x = b to 1e-8: FP32 inner CG with
FP64 reliable updates and FP64 solution accumulation, source and solution
resident on the device.  The JSON line also carries the plain FP64 GPU CG on
the same problem (same kernel template), the Dslash throughput per storage
format, the 16-bit mixed solve, the HBM roofline of the dominant kernel, the
end-to-end time through the C ABI with host buffers, the CPU oracle baseline
and the SM clocks seen during the timed region.

``--impl reference`` times the CPU oracle instead (the reference arm).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = 'CG time-to-1e-8 & Dslash GB/s at 20^3x64 vs FP64 CG; serve p50/p99 latency'
DIMS = (20, 20, 20, 64)
EPS, GAUGE_SEED, SRC_SEED, MASS, TOL = 0.25, 0, 0, 0.01, 1e-8
# Algorithmic bytes per output site of one Dslash: 16 links + 1 input + 1 output
# colour vector (neighbour gathers hit L2).
DSLASH_BYTES = {('f64', 18): 2400, ('f64', 12): 2016, ('f32', 18): 1200, ('f32', 12): 1008,
                ('i16', 18): 608, ('i16', 12): 512}
DSLASH_FLOPS = 1146
# Algorithmic bytes per output site of the CG's two FP32 18-real kernels:
# D_oe p with <p, A p>: links 1152 + p in 24 + t out 24 (the own-site p is
# the same input field); D_eo t with the update: links 1152 + t 24 + p 24 +
# r in/out 48 + xs in/out 48.  The separate xpay kernel moves 72 B per site.
CG_KERNEL_BYTES = {'cg_oe': 1200, 'cg_eo': 1296}
CG_FLOPS_PER_SITE_ITER = 2364
PAPER_CONTEXT_GFLOPS = 46.48   # mixed-precision CG, GTX Titan Black (Table 2)
# DRAM traffic (read + write) of one launch of the CG's D_eo kernel with the
# update (FP32, 18-real, 1 RHS, mode 4) at 20^3 x 64 from an ncu capture of
# the kernel sources with this fingerprint (dram__bytes_read.sum +
# dram__bytes_write.sum; profiles/cg_kernels_20x64.md).  A changed source
# reports traffic null until it is captured again.
NCU_TRAFFIC = {'fingerprint': '652356ae17618aff', 'bytes_per_launch': 324.3e6}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument('--gpus', type=int, default=1)
    p.add_argument('--steps', type=int, default=5)
    p.add_argument('--warmup', type=int, default=3)
    p.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    p.add_argument('--cpu-sample-s', type=float, default=15.0,
                   help='seconds of oracle work in the CPU baseline sample')
    p.add_argument('--no-cpu-baseline', action='store_true')
    p.add_argument('--dslash-iters', type=int, default=200)
    p.add_argument('--serve-requests', type=int, default=2000,
                   help='requests in the serving run (0: skip it)')
    p.add_argument('--no-extra', action='store_true',
                   help='skip the 32^3x64 16-bit and 24^3x64 batched workloads')
    p.add_argument('--dslash-only', default=None, metavar='FORMATS',
                   help='profiling aid: only time the Dslash in these formats '
                        '(comma list of prec_recon, e.g. f32_18), no solves')
    p.add_argument('--dims', default=None, metavar='LX,LY,LZ,LT',
                   help='lattice of the --dslash-only / --npr-only run (default 20,20,20,64)')
    p.add_argument('--npr-only', action='store_true',
                   help='profiling aid: only run the NPR four-fermion workload')
    p.add_argument('--npr-reps', type=int, default=3)
    p.add_argument('--fatten-only', action='store_true',
                   help='profiling aid: only time the two GPU link fattenings (--dims)')
    p.add_argument('--batched-only', action='store_true',
                   help='profiling aid: only run the 24^3x64 multi-RHS / multi-shift workload')
    p.add_argument('--batched-dslash-only', action='store_true',
                   help='profiling aid: only time the 12-system Dslash kernels at 24^3x64')
    return p.parse_args()


def kernel_fingerprint():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, 'paper_1411_2223_gb300', 'csrc')
    for f in ('dslash.cuh', 'sq_device.cuh', 'dslash_f32.cu'):
        h.update(open(os.path.join(csrc, f), 'rb').read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    try:
        d = json.load(open(path))
        return float(d['hbm_gbs']), 'measured'
    except Exception:  # noqa: BLE001
        return 6800.0, 'fallback'


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix='.csv')
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.device), '--query-gpu=' + self.FIELDS,
                 '--format=csv,noheader,nounits', '-lms', '200'],
                stdout=open(self.path, 'w'), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(',')]
                if len(f) >= 9 and f[1].replace('.', '').isdigit():
                    rows.append(f)
        except Exception:  # noqa: BLE001
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['unavailable'], 'samples': 0}
        sm = [float(r[1]) for r in rows]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == 'Active'})
        loaded = [s for s, r in zip(sm, rows) if float(r[3] or 0) > 200.0] or sm
        return {'sm_mhz': statistics.median(loaded), 'sm_max_mhz': float(rows[0][2]),
                'reasons': reasons, 'samples': len(rows),
                'power_w_max': max(float(r[3] or 0) for r in rows)}


# ------------------------------------------------------------------- CPU oracle

def cpu_baseline(fat, lng, b, sample_s):
    """Oracle FP64 CG on the host cores: a bounded number of iterations on the
    full workload, extrapolated to the oracle's own iteration count to 1e-8
    (stored by tests/golden/make_golden.py, which runs only the oracle)."""
    import oracle
    gold = json.load(open(os.path.join(ROOT, 'tests', 'golden', 'oracle_cg.json')))
    iters_full = gold['cg_20x20x20x64_m0.01_tol1e-8']['iterations']
    t0 = time.time()
    oracle.cg(DIMS, fat, lng, MASS, b, TOL, max_iter=2)
    per_iter = (time.time() - t0) / 3.0          # 2 iterations + final true residual
    n = max(2, min(200, int(sample_s / max(per_iter, 1e-3))))
    t0 = time.time()
    oracle.cg(DIMS, fat, lng, MASS, b, TOL, max_iter=n)
    el = time.time() - t0
    per_iter = el / (n + 1)
    cores = int(os.environ.get('OMP_NUM_THREADS', os.cpu_count() or 1))
    return {'value': per_iter * iters_full * 1e3, 'unit': 'ms', 'cores': cores, 'kind': 'oracle',
            'sample': '%d oracle FP64 CG iterations on the 20^3x64 workload (%.1f s), scaled by '
                      'the oracle\'s %d iterations to 1e-8' % (n, el, iters_full),
            'ms_per_iteration': per_iter * 1e3}


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores.  A step is a
    bounded sample of the workload -- n oracle FP64 CG iterations on the
    20^3 x 64 system, n chosen so that the warm-up and timed steps take about
    90 s -- so ms_per_step is the measured time of a step.  `value`, in the
    metric's unit (ms to solve to 1e-8), is one complete oracle solve to
    1e-8, timed after the steps; the per-iteration extrapolation is kept as
    a labelled extra."""
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    import oracle
    import synth
    fat, lng = synth.gauge_field(DIMS, EPS, GAUGE_SEED)
    b = synth.gaussian_source(int(np.prod(DIMS)) // 2, SRC_SEED)
    t0 = time.time()
    oracle.cg(DIMS, fat, lng, MASS, b, TOL, max_iter=2)
    per_iter = (time.time() - t0) / 3.0          # 2 iterations + the final true residual
    n = max(1, int(90.0 / (args.warmup + args.steps) / per_iter) - 1)
    step_ms = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.cg(DIMS, fat, lng, MASS, b, TOL, max_iter=n)
        dt = (time.perf_counter() - t0) * 1e3
        if k >= args.warmup:
            step_ms.append(dt)
    ms_step = statistics.median(step_ms)
    t0 = time.perf_counter()
    _, iters, res = oracle.cg(DIMS, fat, lng, MASS, b, TOL)
    full_ms = (time.perf_counter() - t0) * 1e3
    cores = int(os.environ.get('OMP_NUM_THREADS', os.cpu_count() or 1))
    sample = ('a step is %d oracle FP64 CG iterations (+ the final FP64 residual) on the '
              '20^3x64 workload; value is one complete oracle solve to 1e-8 (%d iterations, '
              'residual %.2e), timed' % (n, iters, res))
    line = {'impl': 'reference', 'metric': METRIC, 'value': round(full_ms, 1), 'unit': 'ms',
            'n_gpus': args.gpus, 'steps': args.steps, 'warmup': args.warmup,
            'ms_per_step': round(ms_step, 1), 'step': '%d oracle CG iterations' % n,
            'higher_is_better': False, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic', 'config': config_dict(),
            'cpu_baseline': {'value': round(full_ms, 1), 'unit': 'ms', 'cores': cores,
                             'kind': 'oracle', 'sample': sample,
                             'extrapolated_from_steps_ms': round(ms_step / (n + 1) * iters, 1)},
            'e2e': {'value': round(full_ms, 1), 'unit': 'ms', 'h2d_bytes_per_step': 0,
                    'd2h_bytes_per_step': 0}}
    print(json.dumps(line))
    return 0


def config_dict():
    return {'workload': 'asqtad even-odd CG 20^3x64 (eps 0.25 synthetic links, seed 0), '
                        'am 0.01, tol 1e-8, 1 RHS, FP32 inner CG + FP64 reliable updates',
            'lattice': 'x'.join(map(str, DIMS)), 'mass': MASS, 'tol': TOL, 'rhs': 1,
            'l2': 'inputs larger than L2: FP32 links 295 MB per parity, both parities per '
                  'iteration; Dslash timing alternates parities',
            'parallelism': 'replicas'}


# ------------------------------------------------------------------- GPU arm

# Serving workload: volumes drawn uniformly from four resident gauge fields
# (seeds 1..4), am ~ U[0.005, 0.05], tol in {1e-6, 1e-8}; a pool of eight
# Gaussian sources per field (seed 10000*field + k) is cycled through.
SERVE_FIELDS = [((8, 8, 8, 8), 1), ((16, 16, 16, 32), 2), ((20, 20, 20, 64), 3),
                ((24, 24, 24, 48), 4)]


def serve_bench(ctx, n_req, sq):
    """Closed-loop throughput (32 clients), then Poisson arrivals at 0.8x and
    0.5x that rate, and the FP64 error of a sample of served solutions."""
    import numpy as np
    import synth
    flags = sq.GAUGE_NO_I16 | sq.GAUGE_NO_LONG12
    gids, pools = [], []
    for dims, seed in SERVE_FIELDS:
        fat, lng = synth.gauge_field(dims, EPS, seed)
        gids.append(ctx.gauge_load(dims, fat, lng, flags=flags))
        vh = int(np.prod(dims)) // 2
        pools.append([synth.gaussian_source(vh, 10000 * seed + k) for k in range(8)])
        del fat, lng
    rng = np.random.default_rng(7)
    reqs = [(int(f), float(m), float(t)) for f, m, t in
            zip(rng.integers(0, 4, n_req), rng.uniform(0.005, 0.05, n_req),
                np.array([1e-6, 1e-8])[rng.integers(0, 2, n_req)])]
    ctx.serve_configure(slots_per_batch=8, block_iters=8)

    def submit(i):
        f, m, t = reqs[i]
        return ctx.serve_submit(gids[f], pools[f][i % 8], m, t)

    # warm-up: tuning and graph capture of every field's batch
    for t in [ctx.serve_submit(g, pools[k][0], 0.02, 1e-6) for k, g in enumerate(gids)]:
        ctx.serve_poll(t, timeout_us=-1, want_x=False)
    ctx.serve_stats(reset=True)
    # closed loop: as many clients as slots (4 fields x 8), each submitting
    # its next request when its previous one has returned
    from collections import deque
    clients = 4 * 8
    t0 = time.time()
    inflight = deque(submit(i) for i in range(min(clients, n_req)))
    nxt, bad = len(inflight), 0
    while inflight:
        bad += ctx.serve_poll(inflight.popleft(), timeout_us=-1, want_x=False)[0] != 0
        if nxt < n_req:
            inflight.append(submit(nxt))
            nxt += 1
    closed_s = time.time() - t0
    closed = ctx.serve_stats(reset=True)

    def open_loop(load, n):
        """Poisson arrivals at `load` x the closed-loop rate, n requests."""
        rate = load * n_req / closed_s
        gaps = rng.exponential(1.0 / rate, n)
        done = []
        tks = []
        t0 = time.time()
        due = t0
        for i in range(n):
            due += gaps[i]
            dt = due - time.time()
            if dt > 0:
                time.sleep(dt)
            tks.append(submit(i))
        for t in tks:
            done.append(ctx.serve_poll(t, timeout_us=-1, want_x=False)[0])
        secs = time.time() - t0
        st = ctx.serve_stats(reset=True)
        return ({'load': load, 'arrival_rate_hz': round(rate, 2), 'requests': n,
                 'seconds': round(secs, 2), 'p50_ms': round(st['p50_ms'], 2),
                 'p99_ms': round(st['p99_ms'], 2), 'mean_ms': round(st['mean_ms'], 2),
                 'solves_per_s': round(st['solves_per_s'], 2)},
                sum(x != 0 for x in done))
    opened, b1 = open_loop(0.8, n_req)
    half, b2 = open_loop(0.5, n_req // 2)
    bad += b1 + b2
    # FP64 error of served solutions: the first two requests of each field,
    # served again and compared with the plain FP64 GPU CG of the same system
    sample = []
    for f in range(4):
        for i in [k for k in range(n_req) if reqs[k][0] == f][:2]:
            _, m, t = reqs[i]
            src = pools[f][i % 8]
            vh = src.shape[0]
            status, x, stx = ctx.serve_poll(submit(i), vh=vh, timeout_us=-1)
            x64, _ = ctx.cg_solve(gids[f], src, m, 1e-10, precision='f64')
            sample.append({'lattice': 'x'.join(map(str, SERVE_FIELDS[f][0])), 'mass': round(m, 5),
                           'tol': t, 'status': status, 'true_residual': stx['true_residual'],
                           'fp64_error_vs_fp64_cg': float(np.linalg.norm(x - x64) /
                                                          np.linalg.norm(x64))})
    for g in gids:
        ctx.gauge_free(g)
    return {'requests': n_req, 'failed': int(bad),
            'workload': 'volumes uniform over 8^4, 16^3x32, 20^3x64, 24^3x48 (4 resident '
                        'fields), am ~ U[0.005,0.05], tol in {1e-6,1e-8}, 8 slots per field, '
                        'FP32 CG + FP64 reliable updates',
            'closed_loop': {'clients': clients, 'solves_per_s': round(n_req / closed_s, 2),
                            'p50_ms': round(closed['p50_ms'], 2),
                            'p99_ms': round(closed['p99_ms'], 2)},
            'fp64_error_sample': sample,
            'open_loop': opened, 'open_loop_half_load': half}


# 16-bit workload: 32^3 x 64, eps 0.25, am 0.01, tol 1e-8, 16-bit storage with
# per-site norms, 12-real long links, FP32 accumulation, FP64 reliable updates.
I16_DIMS = (32, 32, 32, 64)
# Batched workload: 24^3 x 64, eps 0.25; 12 Gaussian sources (seeds 0..11) at
# am 0.01 in one multi-RHS solve, and 8 masses am = 0.005 * 20^(i/7) from one
# source (seed 0) in one multi-shift solve; tol 1e-8, FP32 + FP64 reliable updates.
BATCH_DIMS = (24, 24, 24, 64)
BATCH_NRHS = 12


def timed(fn, stream, reps=1):
    """Device time per call of fn (CUDA events on `stream`) and fn's last result."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps, out


def i16_workload(ctx, sq, stream, dslash_iters):
    """32^3 x 64 in 16-bit storage: solve time, FP64 error against the plain
    FP64 GPU CG solution, and the 16-bit Dslash throughput at this volume."""
    import numpy as np
    import torch
    import synth
    dims = I16_DIMS
    vh = int(np.prod(dims)) // 2
    fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
    gid = ctx.gauge_load(dims, fat, lng, flags=sq.GAUGE_NO_F32)
    del fat, lng
    b = torch.from_numpy(synth.gaussian_source(vh, SRC_SEED)).cuda()
    x = torch.empty_like(b)

    def solve(prec, recon):
        return ctx.cg_solve(gid, b, MASS, TOL, precision=prec, long_recon=recon, stream=stream,
                            out=x)[1]
    solve('i16', 12)
    ms16, st16 = timed(lambda: solve('i16', 12), stream, 2)
    x16 = x.clone()
    ms64, st64 = timed(lambda: solve('f64', 18), stream, 1)
    err_same_tol = fp64_error(x16, x)  # against the FP64 CG to the same tol
    ctx.cg_solve(gid, b, MASS, 1e-10, precision='f64', stream=stream, out=x)
    err = fp64_error(x16, x)
    dsl = time_dslash(ctx, gid, b, stream, vh, (('i16', 12), ('i16', 18)), dslash_iters)
    ctx.gauge_free(gid)
    return {'workload': '32^3x64 (eps 0.25 synthetic links, seed 0), am 0.01, tol 1e-8, 16-bit '
                        'storage + per-site norms, 12-real long links, FP32 accumulate, FP64 '
                        'reliable updates',
            'ms': round(ms16, 3), 'iterations': st16['iterations'],
            'reliable_updates': st16['reliable_updates'],
            'true_residual': st16['true_residual'],
            'fp64_cg_ms': round(ms64, 3), 'fp64_cg_iterations': st64['iterations'],
            'speedup_vs_fp64': round(ms64 / ms16, 3),
            'fp64_error_vs_fp64_cg': err,
            'fp64_error_vs_fp64_cg_same_tol': err_same_tol, 'dslash': dsl}


def fp64_peak_tflops():
    """Measured FP64 throughput of this GPU (cuBLAS DGEMM through torch, best
    of 3): the denominator of the FP64-bound kernels' rooflines."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device='cuda')
    b = torch.randn(n, n, dtype=torch.float64, device='cuda')
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * n ** 3 / best / 1e12


def fatten_workload(ctx, stream, dims=DIMS):
    """The two GPU link fattenings of the lattice's thin links (eps 0.25,
    seed 0): the workloads' recipe and MILC's asqtad path set, FP64."""
    import numpy as np
    import torch
    import synth
    vol = int(np.prod(dims))
    lat = 'x'.join(map(str, dims))
    thin = torch.from_numpy(synth.thin_links(dims, EPS, GAUGE_SEED)).cuda()
    f, l = torch.empty_like(thin), torch.empty_like(thin)
    ctx.gauge_fatten(dims, thin, f, l, stream=stream)
    ms_f, _ = timed(lambda: ctx.gauge_fatten(dims, thin, f, l, stream=stream), stream, 5)
    ctx.gauge_fatten_asqtad(dims, thin, f, l, stream=stream)
    ms_a, _ = timed(lambda: ctx.gauge_fatten_asqtad(dims, thin, f, l, stream=stream), stream, 2)
    # asqtad by nested staple fields: 2 SU(3) products per staple, 6 three-
    # link, 6 Lepage, 24 five-link and 48 seven-link staples, 2 for the Naik
    # link (216 flops each); 60 scaled accumulations of 18 reals (36 flops),
    # 24 sums of two seven-link staples (18) and the one-link term (18)
    flops_a = 4 * vol * (170 * 216 + 60 * 36 + 24 * 18 + 18)
    # flops per link: 6 staples x 2 products + Naik 2 products, 3x3 complex
    # product = 27 complex multiply-adds = 216 real flops; plus the sums
    flops = 4 * vol * (14 * 216 + 6 * 18 + 36)
    peak = fp64_peak_tflops()
    gfl = flops / (ms_f * 1e-3) / 1e9
    return {'fatten_asqtad': {'workload': '%s thin links (eps 0.25, seed 0) -> asqtad fat '
                                          'links (MILC path set: 1-link, 6 3-link, 24 5-link, '
                                          '48 7-link staples, 6 Lepage, built as nested staple '
                                          'fields) and Naik links, FP64' % lat,
                              'ms': round(ms_a, 3),
                              'gflops_fp64': round(flops_a / (ms_a * 1e-3) / 1e9, 1),
                              'frac_of_fp64_peak': round(flops_a / (ms_a * 1e-3) / 1e12 / peak,
                                                         4)},
            'fatten': {'workload': '%s thin links (eps 0.25, seed 0) -> fat (6 staples) and '
                                   'long links, FP64' % lat,
                       'ms': round(ms_f, 3), 'gflops_fp64': round(gfl, 1),
                       'roofline': {'bound': 'alu', 'achieved': round(gfl / 1e3, 4),
                                    'peak': round(peak, 4), 'unit': 'TFLOP/s',
                                    'frac': round(gfl / 1e3 / peak, 4),
                                    'peak_kind': 'measured FP64 DGEMM (torch.matmul 4096^3)'}}}


def full_lattice_workload(ctx, sq, stream, fat, lng):
    """The whole-lattice solve (m + D) x = b at 20^3 x 64 (even-odd CG, and
    BiCGstab for comparison) and the GPU link fattening of the same lattice's
    thin links."""
    import numpy as np
    import torch
    dims = DIMS
    vol = int(np.prod(dims))
    gid = ctx.gauge_load(dims, fat, lng, flags=sq.GAUGE_NO_I16 | sq.GAUGE_NO_LONG12)
    g = np.random.default_rng(SRC_SEED).standard_normal((vol, 3, 2))
    b = torch.from_numpy(g[..., 0] + 1j * g[..., 1]).cuda()
    ctx.cg_solve_full(gid, b, MASS, TOL, stream=stream)
    ms, (x, st) = timed(lambda: ctx.cg_solve_full(gid, b, MASS, TOL, stream=stream), stream, 2)
    x64 = ctx.cg_solve_full(gid, b, MASS, 1e-10, precision='f64', stream=stream)[0]
    err_full = fp64_error(x, x64)
    # BiCGstab on M = m + D itself (the BiCG-family comparison solver): FP64,
    # and FP32 with FP64 reliable updates
    ms_b, (_, stb) = timed(lambda: ctx.bicgstab_solve_full(gid, b, MASS, TOL, stream=stream),
                           stream, 1)
    ms_bm, (_, stbm) = timed(lambda: ctx.bicgstab_solve_full(gid, b, MASS, TOL, precision='f32',
                                                             stream=stream), stream, 1)
    ctx.gauge_free(gid)
    return {'solve': {'workload': '20^3x64 whole lattice (m + D) x = b, Gaussian source (seed 0), '
                                  'am 0.01, tol 1e-8: even-site FP32 CG + FP64 reliable updates, '
                                  'odd sites reconstructed',
                      'ms': round(ms, 3), 'iterations': st['iterations'],
                      'full_true_residual': st['true_residual'],
                      'fp64_error_vs_fp64_cg': err_full},
            'bicgstab': {'workload': '20^3x64 whole lattice (m + D) x = b, same source, am 0.01, '
                                     'tol 1e-8: FP64 BiCGstab on M itself',
                         'ms': round(ms_b, 1), 'iterations': stb['iterations'],
                         'm_products': 2 * stb['iterations'],
                         'full_true_residual': stb['true_residual'],
                         'vs_even_odd_cg': round(ms_b / ms, 1)},
            'bicgstab_mixed': {'workload': 'same system: FP32 BiCGstab on M with FP64 reliable '
                                           'updates (delta 0.1)',
                               'ms': round(ms_bm, 1), 'iterations': stbm['iterations'],
                               'reliable_updates': stbm['reliable_updates'],
                               'full_true_residual': stbm['true_residual'],
                               'vs_even_odd_cg': round(ms_bm / ms, 1)},
            **fatten_workload(ctx, stream, dims)}


# Flops of one hypercube of the NPR operator (Eq. 1), counting 8 per complex
# multiply-add of the factored evaluation: averaged links 224 SU(3) products
# (U_AD for A < D at distance >= 2, the recursion over the first step), the
# sandwiches P = G1^dag U G4 and Q = G3^dag U G2 (2 x 256 pairs x 2
# products), and per operator 256 corner pairs x 81 outputs.
def npr_flops_per_hypercube(nops):
    return 8 * (224 * 27 + 2 * 256 * 2 * 27 + 256 * 81 * nops)


NPR_PAPER_GFLOPS = 113.36   # NPR four-fermion part, GTX Titan Black, 1 GPU (Table 3)


def npr_workload(ctx, stream, dims=DIMS, reps=3):
    """The NPR one-colour four-fermion operator (Eq. 1) over the 20^3 x 64
    lattice: thin links (eps 0.25, seed 0), four Gaussian propagators (seed 1),
    the 8 B_K-basis operators; sums over hypercubes only (no per-hypercube
    output).  FP64 throughput against the measured DGEMM rate.  Returns the
    result and the host inputs (for the CPU baseline)."""
    import numpy as np
    import torch
    import synth
    from synth import npr as snpr
    vol = int(np.prod(dims))
    nhc = vol // 16
    links = synth.thin_links(dims, EPS, GAUGE_SEED)
    props = snpr.propagators(dims, 1)
    ops = snpr.bk_ops()
    u = torch.from_numpy(links).cuda()
    ps = [torch.from_numpy(p).cuda() for p in props]
    out = torch.empty((len(ops), 3, 3, 3, 3), dtype=torch.complex128, device='cuda')
    with torch.cuda.stream(stream):
        ctx.npr_four_fermion(dims, u, ps, ops, out, stream=stream)
        ms, _ = timed(lambda: ctx.npr_four_fermion(dims, u, ps, ops, out, stream=stream),
                      stream, reps)
    flops = npr_flops_per_hypercube(len(ops)) * nhc
    tflops = flops / (ms * 1e-3) / 1e12
    peak = fp64_peak_tflops()
    res = {'workload': '%s NPR one-colour four-fermion operator (Eq. 1), FP64: thin links '
                       '(eps 0.25, seed 0), 4 Gaussian propagators (seed 1), 8 B_K-basis '
                       'operators, summed over %d hypercubes' % ('x'.join(map(str, dims)), nhc),
           'ms': round(ms, 3), 'gflops_fp64': round(tflops * 1e3, 1),
           'flops_per_hypercube': npr_flops_per_hypercube(len(ops)),
           'roofline': {'bound': 'alu', 'achieved': round(tflops, 4), 'peak': round(peak, 4),
                        'unit': 'TFLOP/s', 'frac': round(tflops / peak, 4),
                        'peak_kind': 'measured FP64 DGEMM (torch.matmul 4096^3)'},
           'paper_context': {'gflops_titan_black_1gpu': NPR_PAPER_GFLOPS,
                             'note': 'Table 3; different hardware and flop convention'}}
    return res, (dims, links, props, ops)


def npr_cpu_baseline(inputs, n_hc=4096):
    """The oracle's NPR operator on the host cores for the first n_hc
    hypercubes of the workload, scaled to the whole lattice."""
    import oracle
    dims, links, props, ops = inputs
    nhc = (dims[0] * dims[1] * dims[2] * dims[3]) // 16
    t0 = time.perf_counter()
    oracle.npr_four_fermion(dims, links, props, ops, hypercubes=list(range(n_hc)))
    dt = time.perf_counter() - t0
    return {'value': round(dt * 1e3 * nhc / n_hc, 1), 'unit': 'ms', 'cores': os.cpu_count(),
            'kind': 'oracle',
            'sample': '%d of %d hypercubes x %d operators (%.1f s), scaled to the lattice'
                      % (n_hc, nhc, len(ops), dt)}


def fp64_error(x, x64):
    """|x - x64| / |x64| (device tensors)."""
    import torch
    return float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))


def batched_dslash(ctx, sq, dims, stream, nrhs=BATCH_NRHS):
    """The FP32 18-real Dslash on 12 right-hand sides in one launch
    (dslash_apply_multi) at the tuner's tile, and the CG's two batched
    kernels (sq_time_dslash): device time per launch against the HBM
    roofline, links counted once per launch plus every system's own
    vectors."""
    import numpy as np
    import torch
    import synth
    vh = int(np.prod(dims)) // 2
    gid = None
    fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
    gid = ctx.gauge_load(dims, fat, lng, flags=sq.GAUGE_NO_I16 | sq.GAUGE_NO_LONG12 |
                         sq.GAUGE_NO_F64)
    del fat, lng
    nbytes, _ = ctx.spinor_bytes(gid, 'f32')
    a = torch.zeros(nrhs * nbytes, dtype=torch.uint8, device='cuda')
    c = torch.zeros_like(a)
    src = torch.from_numpy(synth.gaussian_source(vh, SRC_SEED)).cuda()
    for j in range(nrhs):
        ctx.pack_spinor(gid, 'f32', src, a[j * nbytes:(j + 1) * nbytes], stream)
    iters = 40
    for k in range(4):
        ctx.dslash_apply_multi(gid, k & 1, 'f32', 18, nrhs, a if k & 1 else c,
                               c if k & 1 else a, stream)
    ms, _ = timed(lambda: [ctx.dslash_apply_multi(gid, k & 1, 'f32', 18, nrhs, a if k & 1 else c,
                                                  c if k & 1 else a, stream)
                           for k in range(iters)], stream)
    us = ms * 1e3 / iters
    links = 1152
    peak, kind = measured_peak()
    out = {'plain': {'us': round(us, 2), 'rhs_tile': ctx.tuned_launch(gid, 'f32', 18, nrhs,
                                                                       'plain')[1],
                     'algorithmic_bytes_per_site': links + nrhs * 48,
                     'GBs': round((links + nrhs * 48) * vh / (us * 1e-6) / 1e9, 1)}}
    # the CG's kernels: D_oe with <p, A p> reads p and writes t per system
    # (plus own p), D_eo with the update reads t, p, r, xs and writes r, xs
    for mode, per_sys in (('cg_oe', 72), ('cg_eo', 144)):
        us_m = ctx.time_dslash(gid, 'f32', 18, nrhs, mode, 50, stream)
        b = links + nrhs * per_sys
        out[mode] = {'us': round(us_m, 2),
                     'rhs_tile': ctx.tuned_launch(gid, 'f32', 18, nrhs, mode)[1],
                     'algorithmic_bytes_per_site': b,
                     'GBs': round(b * vh / (us_m * 1e-6) / 1e9, 1)}
    for v in out.values():
        v['frac_of_hbm'] = round(v['GBs'] / peak, 4)
    out['peak_GBs'] = peak
    out['peak_kind'] = kind
    ctx.gauge_free(gid)
    return out


def batched_workload(ctx, sq, stream):
    """24^3 x 64: 12 right-hand sides in one batched solve against 12 single
    solves, and 8 masses in one multi-shift solve against 8 single solves."""
    import numpy as np
    import torch
    import synth
    dims = BATCH_DIMS
    vh = int(np.prod(dims)) // 2
    fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
    gid = ctx.gauge_load(dims, fat, lng, flags=sq.GAUGE_NO_I16 | sq.GAUGE_NO_LONG12)
    del fat, lng
    srcs = torch.from_numpy(synth.gaussian_sources(vh, range(BATCH_NRHS))).cuda()
    xs = torch.empty_like(srcs)
    masses = [MASS] * BATCH_NRHS
    shifts = list(0.005 * 20.0 ** (np.arange(8) / 7.0))

    def multi():
        return ctx.cg_solve_multi(gid, srcs, masses, TOL, stream=stream, out=xs)[1]

    def singles(sources, ms):
        return [ctx.cg_solve(gid, s, m, TOL, stream=stream, out=xs[0])[1]
                for s, m in zip(sources, ms)]

    def mshift():
        return ctx.cg_solve_multishift(gid, srcs[0], shifts, TOL, stream=stream)[1]
    multi()
    ms_multi, st_multi = timed(multi, stream)
    x_multi = xs.clone()
    singles(srcs[:1], masses[:1])
    ms_single, st_single = timed(lambda: singles(srcs, masses), stream)
    mshift()
    ms_shift, st_shift = timed(mshift, stream)
    x_shift = ctx.cg_solve_multishift(gid, srcs[0], shifts, TOL, stream=stream)[0]
    ms_shift_single, _ = timed(lambda: singles([srcs[0]] * len(shifts), shifts), stream)
    # FP64 error of every result against the plain FP64 GPU CG of the same
    # system (batched FP64 solves, to 1e-10)
    ref = ctx.cg_solve_multi(gid, srcs, masses, 1e-10, precision='f64', stream=stream)[0]
    err_multi = [fp64_error(x_multi[j], ref[j]) for j in range(BATCH_NRHS)]
    ref = ctx.cg_solve_multi(gid, srcs[0].expand(len(shifts), -1, -1).contiguous(), shifts,
                             1e-10, precision='f64', stream=stream)[0]
    err_shift = [fp64_error(x_shift[j], ref[j]) for j in range(len(shifts))]
    ctx.gauge_free(gid)
    worst = max(s['true_residual'] for s in st_multi + st_shift)
    return {'workload': '24^3x64 (eps 0.25 synthetic links, seed 0), tol 1e-8, FP32 + FP64 '
                        'reliable updates: 12 sources (seeds 0..11) at am 0.01 batched; 8 masses '
                        'am = 0.005*20^(i/7) multi-shift from source seed 0',
            'multi_rhs': {'rhs': BATCH_NRHS, 'ms': round(ms_multi, 3),
                          'ms_per_solve': round(ms_multi / BATCH_NRHS, 3),
                          'single_solves_ms': round(ms_single, 3),
                          'speedup_vs_single': round(ms_single / ms_multi, 3),
                          'iterations_max': max(s['iterations'] for s in st_multi),
                          'rhs_tile': [st_multi[0]['oe_rhs_tile'], st_multi[0]['eo_rhs_tile']],
                          'fp64_error_vs_fp64_cg': err_multi},
            'multi_shift': {'shifts': len(shifts), 'ms': round(ms_shift, 3),
                            'single_solves_ms': round(ms_shift_single, 3),
                            'speedup_vs_single': round(ms_shift_single / ms_shift, 3),
                            'iterations': [s['iterations'] for s in st_shift],
                            'fp64_error_vs_fp64_cg': err_shift},
            'dslash_12rhs': batched_dslash(ctx, sq, dims, stream),
            'worst_true_residual': worst}


def max_over_ranks(value, dist=None):
    """Slowest replica's value (replicas only: no data-path collective; this
    one all-reduce of a scalar happens after the timed region)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    dev = 'cuda' if dist.get_backend() == 'nccl' else 'cpu'
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_dslash(ctx, gid, b_dev, stream, vh, formats, iters):
    """Average device time per Dslash launch (CUDA events on the launching
    stream), alternating output parities so both link fields stream from HBM."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    bufs = {}
    for prec, recon in formats:
        nbytes, _ = ctx.spinor_bytes(gid, prec)
        if prec not in bufs:
            bufs[prec] = (torch.zeros(nbytes, dtype=torch.uint8, device='cuda'),
                          torch.zeros(nbytes, dtype=torch.uint8, device='cuda'))
            ctx.pack_spinor(gid, prec, b_dev, bufs[prec][0], stream)
            ctx.pack_spinor(gid, prec, b_dev, bufs[prec][1], stream)
        a, c = bufs[prec]
        n_it = iters if prec != 'f64' else max(20, iters // 4)
        for k in range(20):
            ctx.dslash_apply(gid, k & 1, prec, recon, a if k & 1 else c, c if k & 1 else a, stream)
        ev0.record(stream)
        for k in range(n_it):
            ctx.dslash_apply(gid, k & 1, prec, recon, a if k & 1 else c, c if k & 1 else a, stream)
        ev1.record(stream)
        ev1.synchronize()
        us = ev0.elapsed_time(ev1) * 1e3 / n_it
        gbs = DSLASH_BYTES[(prec, recon)] * vh / (us * 1e-6) / 1e9
        out['%s_%d' % (prec, recon)] = {'us': round(us, 2), 'GBs': round(gbs, 1),
                                        'gflops': round(DSLASH_FLOPS * vh / (us * 1e-6) / 1e9, 1)}
    return out


def main():
    args = parse_args()
    if args.impl == 'reference':
        return run_reference(args)
    import numpy as np
    import torch

    import synth
    from paper_1411_2223_gb300 import sq

    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl' if torch.cuda.is_available() else 'gloo')
    torch.cuda.set_device(local)
    dims = DIMS
    if args.dslash_only and args.dims:
        dims = tuple(int(v) for v in args.dims.split(','))
    vh = int(np.prod(dims)) // 2
    if args.batched_dslash_only:
        ctx = sq.Context(local)
        print(json.dumps({'dslash_12rhs': batched_dslash(ctx, sq, BATCH_DIMS,
                                                         torch.cuda.Stream())}))
        ctx.close()
        return 0
    if args.batched_only:
        ctx = sq.Context(local)
        print(json.dumps({'batched_24x64': batched_workload(ctx, sq, torch.cuda.Stream())}))
        ctx.close()
        return 0
    if args.fatten_only:
        fdims = tuple(int(v) for v in args.dims.split(',')) if args.dims else DIMS
        ctx = sq.Context(local)
        print(json.dumps({'fatten': fatten_workload(ctx, torch.cuda.Stream(), fdims)}))
        ctx.close()
        return 0
    if args.npr_only:
        ndims = tuple(int(v) for v in args.dims.split(',')) if args.dims else DIMS
        ctx = sq.Context(local)
        res, _ = npr_workload(ctx, torch.cuda.Stream(), ndims, args.npr_reps)
        print(json.dumps({'npr': res}))
        ctx.close()
        return 0

    fat, lng = synth.gauge_field(dims, EPS, GAUGE_SEED)
    b_host = synth.gaussian_source(vh, SRC_SEED)
    ctx = sq.Context(local)
    gflags = 0
    if args.dslash_only:  # load only the link forms being timed
        want = set(args.dslash_only.split(','))
        if not any(f.startswith('f64') for f in want):
            gflags |= sq.GAUGE_NO_F64
        if not any(f.startswith('f32') for f in want):
            gflags |= sq.GAUGE_NO_F32
        if not any(f.startswith('i16') for f in want):
            gflags |= sq.GAUGE_NO_I16
        if not any(f.endswith('_12') for f in want):
            gflags |= sq.GAUGE_NO_LONG12
    gid = ctx.gauge_load(dims, fat, lng, flags=gflags)
    stream = torch.cuda.Stream()
    b_dev = torch.from_numpy(b_host).cuda()
    x_dev = torch.empty_like(b_dev)
    if args.dslash_only:
        fmts = [(f.split('_')[0], int(f.split('_')[1])) for f in args.dslash_only.split(',')]
        res = time_dslash(ctx, gid, b_dev, stream, vh, fmts, args.dslash_iters)
        print(json.dumps({'dslash': res}))
        ctx.close()
        return 0

    def solve(prec='f32', recon=18, dev=True, out=None):
        if dev:
            return ctx.cg_solve(gid, b_dev, MASS, TOL, precision=prec, long_recon=recon,
                                stream=stream, out=x_dev)
        return ctx.cg_solve(gid, b_host_pinned, MASS, TOL, precision=prec, long_recon=recon,
                            stream=stream, out=x_host_pinned)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # warm-up: tuning, graph capture, first-touch
    for _ in range(args.warmup):
        _, st = solve()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- timed region: K mixed-precision solves, device-resident inputs
    barrier()
    l0 = ctx.kernel_launches()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            _, st = solve()
        ev1.record(stream)
        ev1.synchronize()
    launches = ctx.kernel_launches() - l0
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist)
    iters = st['iterations']
    clk = clocks.summary()

    # ---- plain FP64 GPU CG on the same problem (same kernel template)
    k64 = max(1, min(3, args.steps))
    solve('f64')
    barrier()
    ev0.record(stream)
    for _ in range(k64):
        _, st64 = solve('f64')
    ev1.record(stream)
    ev1.synchronize()
    ms64 = ev0.elapsed_time(ev1) / k64
    x64 = x_dev.clone()

    # ---- 16-bit storage mixed solve (12-real long links)
    solve('i16', 12)
    ev0.record(stream)
    for _ in range(k64):
        _, st16 = solve('i16', 12)
    ev1.record(stream)
    ev1.synchronize()
    ms16 = ev0.elapsed_time(ev1) / k64

    # ---- the same FP32 mixed solve with 12-real (reconstructed) long links
    solve('f32', 12)
    ev0.record(stream)
    for _ in range(k64):
        _, st12 = solve('f32', 12)
    ev1.record(stream)
    ev1.synchronize()
    ms12 = ev0.elapsed_time(ev1) / k64

    # FP64 error of the mixed result: against the plain FP64 GPU CG solution
    # of the same system to 1e-10 (the reference of every error in this
    # report), and against the FP64 CG timed above (tol 1e-8, same Krylov
    # path)
    ctx.cg_solve(gid, b_dev, MASS, 1e-10, precision='f64', stream=stream, out=x_dev)
    x_ref = x_dev.clone()
    solve('f32')
    err = fp64_error(x_dev, x_ref)
    err_same_tol = fp64_error(x_dev, x64)

    # ---- e2e through the C ABI with host buffers (pinned), copies inside
    b_host_pinned = torch.from_numpy(b_host).pin_memory().numpy()
    x_host_pinned = torch.zeros(b_host.shape, dtype=torch.complex128).pin_memory().numpy()
    solve(dev=False)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        solve(dev=False)
    ev1.record(stream)
    ev1.synchronize()
    ms_e2e = ev0.elapsed_time(ev1) / args.steps
    h2d = b_host.nbytes
    d2h = b_host.nbytes

    # ---- Dslash throughput per format (alternating parities: > L2 of links)
    dslash = time_dslash(ctx, gid, b_dev, stream, vh,
                         (('f32', 18), ('f32', 12), ('i16', 12), ('i16', 18), ('f64', 18)),
                         args.dslash_iters)
    peak, peak_kind = measured_peak()
    peak_note = (peak_kind + ' (MEASURED_PEAKS.json hbm_gbs)' if peak_kind == 'measured'
                 else 'fallback')
    # the CG's own kernels at the launch shape the solve uses (CUDA events
    # around back-to-back launches inside the library, on `stream`)
    cg_kernels = {}
    for mode, name in (('cg_oe', 'D_oe p with <p, A p> (mode 3)'),
                       ('cg_eo', 'D_eo t with the m^2 epilogue and the update (mode 4)')):
        us = ctx.time_dslash(gid, 'f32', 18, 1, mode, 200, stream)
        gbs = CG_KERNEL_BYTES[mode] * vh / (us * 1e-6) / 1e9
        cg_kernels[mode] = {'kernel': name, 'us': round(us, 2),
                            'algorithmic_bytes_per_site': CG_KERNEL_BYTES[mode],
                            'GBs': round(gbs, 1), 'frac': round(gbs / peak, 4)}
    dom = cg_kernels['cg_eo']
    traffic = None
    if NCU_TRAFFIC['fingerprint'] == kernel_fingerprint():
        traffic = NCU_TRAFFIC['bytes_per_launch']
    roofline = {'bound': 'hbm', 'achieved': dom['GBs'], 'peak': peak, 'unit': 'GB/s',
                'frac': dom['frac'], 'traffic': traffic,
                'kernel': 'dslash_kernel<F32,18-real,1 RHS,MODE_UPDATE> (the CG\'s D_eo kernel '
                          'with the m^2 epilogue and the update, %.0f%% of the solve), %d '
                          'algorithmic B/site x %d sites per launch'
                          % (100 * dom['us'] / (dom['us'] + cg_kernels['cg_oe']['us'] + 4.0),
                             CG_KERNEL_BYTES['cg_eo'], vh),
                'us_per_launch': dom['us'], 'peak_kind': peak_note}
    us_it = ms * 1e3 / iters
    it_bytes = (CG_KERNEL_BYTES['cg_oe'] + CG_KERNEL_BYTES['cg_eo'] + 72) * vh
    cg_iteration = {'bytes_per_iteration': it_bytes, 'us_per_iteration': round(us_it, 2),
                    'GBs': round(it_bytes / (us_it * 1e-6) / 1e9, 1),
                    'frac': round(it_bytes / (us_it * 1e-6) / 1e9 / peak, 4),
                    'note': 'whole solve time / iterations (init, reliable updates and the '
                            'final residual included); bytes: D_oe %d + D_eo %d + xpay 72 B '
                            'per site' % (CG_KERNEL_BYTES['cg_oe'], CG_KERNEL_BYTES['cg_eo'])}

    serve = serve_bench(ctx, args.serve_requests, sq) if args.serve_requests > 0 else None
    extra_i16 = extra_batch = extra_full = extra_npr = None
    if not args.no_extra:
        ctx.gauge_free(gid)
        extra_npr, npr_inputs = npr_workload(ctx, stream)
        extra_full = full_lattice_workload(ctx, sq, stream, fat, lng)
        extra_i16 = i16_workload(ctx, sq, stream, args.dslash_iters)
        extra_batch = batched_workload(ctx, sq, stream)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(fat, lng, b_host, args.cpu_sample_s)
        if extra_npr is not None:
            cb['npr_20x64'] = npr_cpu_baseline(npr_inputs)

    if rank == 0:
        gflops = CG_FLOPS_PER_SITE_ITER * vh * iters / (ms * 1e-3) / 1e9
        line = {
            'metric': METRIC, 'value': round(ms, 3), 'unit': 'ms', 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': round(ms, 3),
            'higher_is_better': False, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32',
            'data': 'synthetic', 'config': config_dict(),
            'iterations': iters, 'reliable_updates': st['reliable_updates'],
            'true_residual': st['true_residual'], 'cg_gflops': round(gflops, 1),
            'fp64_cg': {'ms': round(ms64, 3), 'iterations': st64['iterations'],
                        'true_residual': st64['true_residual']},
            'speedup_vs_fp64': round(ms64 / ms, 3),
            'fp64_error_vs_fp64_cg': err,
            'fp64_error_vs_fp64_cg_same_tol': err_same_tol,
            'f32_long12_cg': {'ms': round(ms12, 3), 'iterations': st12['iterations'],
                              'reliable_updates': st12['reliable_updates'],
                              'true_residual': st12['true_residual'],
                              'note': 'same FP32 inner CG, Naik links stored as 12 reals '
                                      '(c3 SU(3) reconstructed), fat links 18 reals'},
            'i16_cg': {'ms': round(ms16, 3), 'iterations': st16['iterations'],
                       'reliable_updates': st16['reliable_updates'],
                       'true_residual': st16['true_residual'], 'long_recon': 12},
            'dslash': dslash,
            'serve': serve,
            'i16_32x64': extra_i16,
            'batched_24x64': extra_batch,
            'whole_lattice_20x64': extra_full,
            'npr_20x64': extra_npr,
            'roofline': roofline,
            'cg_kernels': cg_kernels,
            'cg_iteration': cg_iteration,
            'e2e': {'value': round(ms_e2e, 3), 'unit': 'ms', 'h2d_bytes_per_step': h2d,
                    'd2h_bytes_per_step': d2h},
            'gpu_launches': launches,
            'clocks': clk,
            'cpu_baseline': cb,
            'paper_context': {'gflops_mixed_cg_titan_black': PAPER_CONTEXT_GFLOPS,
                              'note': 'Table 2; different hardware and flop convention'},
        }
        print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == '__main__':
    sys.exit(main())
