// Driver of the batched mixed-precision CG (one system per slot).
//
// One iteration is three sloppy kernels and two scalar steps, gated on
// device-resident slot state so that no host decision sits inside an
// iteration:
//   1. t = D_oe p, partials of <p, A p> = m^2 |p|^2 + |t|^2   (sloppy Dslash)
//      F. sum of the partials: alpha                  (one block per system)
//   2. Ap = m^2 p - D_eo t (in registers), xs += alpha p, r -= alpha Ap,
//      partials of |r|^2                              (sloppy Dslash + epilogue)
//      F. sum: beta, or flag a reliable update         (one block per system)
//   3. p = a r + beta p
// (<p, A p> = |M p|^2 with M p = (m p, D_oe p), as D_eo = -D_oe^dag.)
// and after every RU_PERIOD-th iteration (a checkpoint) the reliable-update
// pair, which does work only for flagged slots:
//   R1. t64 = D_oe (x64 + xs)               (FP64 Dslash)
//   R2. x64 += xs, xs = 0; r = b - (m^2 x64 - D_eo t64), |r|^2, <r, p>
//                                           (FP64 Dslash + epilogue; finishes it)
// Checkpoints keep the FP64 kernels' launch cost off most iterations; a slot
// that wants to stop waits frozen for the next checkpoint, so no iteration is
// wasted.  k iterations are captured once into a CUDA graph and replayed; the
// host reads the slot states after each replay.  Finished slots make every
// kernel skip their work, so overshooting the last block costs launches only.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "sq_host.h"

namespace sq {

CGWork::~CGWork() {
  if (exec) cudaGraphExecDestroy(exec);
  if (slots_h) cudaFreeHost(slots_h);
  if (ctx) {
    void *bufs[] = {x64, b64, t64, r, p, t, xs, slots_d, partial, counters};
    for (void *b : bufs)
      if (b) cudaFree(b);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->in_use -= bytes;
  }
  if (gf) gf->users--;
}

int cg_work_create(sq_ctx *ctx, GaugeField *gf, int prec, int recon, int nrhs, CGWork **out) {
  if (!gf->has(prec, recon) || !gf->has(PREC_F64, 18)) return SQ_ERR_UNSUPPORTED;
  std::unique_ptr<CGWork> w(new CGWork());
  w->gf = gf;
  gf->users++;
  w->prec = prec;
  w->recon = recon;
  w->nrhs = nrhs;
  const Geom &g = gf->g;
  w->f64_fb = spinor_bytes(PREC_F64, g.stride);
  w->fb = spinor_bytes(prec, g.stride);
  w->xs_fb = spinor_bytes(xs_prec(prec), g.stride);
  w->partial_stride = (size_t)3 * nrhs * red_stride(g);
  w->counter_stride = (size_t)nrhs * ticket_stride(g);
  size_t sizes[] = {w->f64_fb * nrhs, w->f64_fb * nrhs, w->f64_fb * nrhs, w->fb * nrhs,
                    w->fb * nrhs,     w->fb * nrhs,     w->xs_fb * nrhs,
                    sizeof(SlotState) * nrhs, sizeof(double) * 4 * w->partial_stride,
                    sizeof(unsigned) * 4 * w->counter_stride};
  char **ptrs[] = {&w->x64, &w->b64, &w->t64, &w->r, &w->p, &w->t, &w->xs};
  size_t total = 0;
  for (size_t s : sizes) total += s;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->in_use + total > ctx->budget) return SQ_ERR_OOM;
    ctx->in_use += total;
  }
  w->ctx = ctx;
  w->bytes = total;
  for (int k = 0; k < 7; ++k) SQ_CUDA_TRY(cudaMalloc((void **)ptrs[k], sizes[k]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->slots_d, sizes[7]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->partial, sizes[8]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->counters, sizes[9]));
  SQ_CUDA_TRY(cudaMemset(w->counters, 0, sizes[9]));
  SQ_CUDA_TRY(cudaMemset(w->partial, 0, sizes[8]));
  // vectors start zeroed so no kernel reads NaN garbage from padding
  for (int k = 0; k < 7; ++k) SQ_CUDA_TRY(cudaMemset(*ptrs[k], 0, sizes[k]));
  SQ_CUDA_TRY(cudaMallocHost((void **)&w->slots_h, sizes[7]));
  for (int k = 0; k < nrhs; ++k) {
    std::memset(&w->slots_h[k], 0, sizeof(SlotState));
    w->slots_h[k].status = SLOT_IDLE;
  }
  *out = w.release();
  return SQ_OK;
}

void cg_slot_setup(CGWork *w, int slot, double mass, double tol, double delta, int max_iter) {
  SlotState &s = w->slots_h[slot];
  std::memset(&s, 0, sizeof(s));
  s.m2 = mass * mass;
  s.tol2 = tol * tol;
  s.delta = (w->prec == PREC_F64) ? 0.0 : delta;
  s.max_iter = max_iter;
  s.status = SLOT_INIT;
  s.a_re = 1.0;
}

int cg_slots_upload(CGWork *w, cudaStream_t st) {
  SQ_CUDA_TRY(cudaMemcpyAsync(w->slots_d, w->slots_h, sizeof(SlotState) * w->nrhs,
                              cudaMemcpyHostToDevice, st));
  return SQ_OK;
}

int cg_slots_download(CGWork *w, cudaStream_t st) {
  SQ_CUDA_TRY(cudaMemcpyAsync(w->slots_h, w->slots_d, sizeof(SlotState) * w->nrhs,
                              cudaMemcpyDeviceToHost, st));
  return SQ_OK;
}

static VecArgs vec_args(CGWork *w, int region) {
  VecArgs a;
  a.g = w->gf->g;
  a.nrhs = w->nrhs;
  a.x64 = w->x64;
  a.b64 = w->b64;
  a.f64_fb = w->f64_fb;
  a.r = w->r;
  a.p = w->p;
  a.fb = w->fb;
  a.xs = w->xs;
  a.xs_fb = w->xs_fb;
  a.slots = w->slots_d;
  a.partial = w->partial + region * w->partial_stride;
  a.counter = w->counters + region * w->counter_stride;
  a.checkpoint = 0;
  return a;
}

static DslashArgs dslash_args(CGWork *w, int prec, int recon, int out_parity) {
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = w->gf->g;
  a.out_parity = out_parity;
  a.links = w->gf->link_ptr(prec, recon, out_parity);
  a.ls = w->gf->scales(prec, recon);
  a.nrhs = w->nrhs;
  a.slots = w->slots_d;
  return a;
}

static int check_launch(sq_ctx *ctx, int rc, int nkernels = 1) {
  if (rc != 0) return SQ_ERR_ARG;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "kernel launch", __FILE__, __LINE__);
    return SQ_ERR_CUDA;
  }
  ctx->launches += nkernels;
  return SQ_OK;
}

int cg_enqueue_init(CGWork *w, int guess, cudaStream_t st) {
  VecArgs va = vec_args(w, 3);
  int rc = check_launch(w->ctx, launch_cg_init(w->prec, va, guess, st));
  if (rc) return rc;
  if (guess) {
    if ((rc = cg_enqueue_ru(w, st))) return rc;
    if ((rc = cg_enqueue_xpay(w, st))) return rc;
  }
  return SQ_OK;
}

// The pair has work at few checkpoints: its kernels take a grid of a few
// blocks per SM that loop over the work items of the systems with a pending
// update, so that a checkpoint without one costs a wave of blocks (one block
// per item: 2000 empty blocks per kernel at 20^3 x 64, 41472 for 12 systems
// at 24^3 x 64).
static int ru_grid(const CGWork *w) { return GATED_BLOCKS_PER_SM * w->ctx->sms; }

int cg_enqueue_ru(CGWork *w, cudaStream_t st) {
  // t64 = D_oe (x64 + xs) in FP64 for slots with a pending reliable update
  DslashArgs a = dslash_args(w, PREC_F64, 18, 1);
  a.max_grid = ru_grid(w);
  a.in = w->x64;
  a.in_fb = w->f64_fb;
  a.xs = w->xs;
  a.xs_fb = w->xs_fb;
  a.xs_prec = xs_prec(w->prec);
  a.out = w->t64;
  a.out_fb = w->f64_fb;
  a.gate = GATE_RU;
  int rc = check_launch(w->ctx, launch_dslash(PREC_F64, 18, w->cfg_ru_plain.nr, MODE_PLAIN,
                                              PREC_F64, a, w->cfg_ru_plain.block, st));
  if (rc) return rc;
  // x64 += xs, xs = 0; r = b - (m^2 x64 - D_eo t64) -> sloppy r ; |r|^2, <r, p>
  DslashArgs b = dslash_args(w, PREC_F64, 18, 0);
  b.in = w->t64;
  b.in_fb = w->f64_fb;
  b.out = w->r;
  b.out_fb = w->fb;
  b.x64 = w->x64;
  b.b64 = w->b64;
  b.f64_fb = w->f64_fb;
  b.xs = w->xs;
  b.xs_fb = w->xs_fb;
  b.xs_prec = xs_prec(w->prec);
  b.ps = w->p;
  b.ps_fb = w->fb;
  b.partial = w->partial + 2 * w->partial_stride;
  b.counter = w->counters + 2 * w->counter_stride;
  b.gate = GATE_RU;
  b.max_grid = ru_grid(w);
  return check_launch(w->ctx, launch_dslash(PREC_F64, 18, w->cfg_ru_resid.nr, MODE_RESID,
                                            w->prec, b, w->cfg_ru_resid.block, st));
}

int cg_enqueue_xpay(CGWork *w, cudaStream_t st) {
  return check_launch(w->ctx, launch_cg_xpay(w->prec, vec_args(w, 1), st));
}

int cg_enqueue_iteration(CGWork *w, cudaStream_t st, int checkpoint) {
  int rc;
  // t = D_oe p, with |t|^2 + m^2 |p|^2 = <p, A p>: alpha
  DslashArgs a = dslash_args(w, w->prec, w->recon, 1);
  a.in = w->p;
  a.in_fb = w->fb;
  a.out = w->t;
  a.out_fb = w->fb;
  a.partial = w->partial;
  a.counter = w->counters;
  a.gate = GATE_RUNNING;
  rc = check_launch(w->ctx, launch_dslash(w->prec, w->recon, w->cfg_norm.nr, MODE_NORM,
                                          w->prec, a, w->cfg_norm.block, st));
  if (rc) return rc;
  if ((rc = check_launch(w->ctx, launch_cg_finish(0, vec_args(w, 0), st)))) return rc;
  // Ap = m^2 p - D_eo t in registers: xs += alpha p, r -= alpha Ap, |r|^2: beta
  DslashArgs b = dslash_args(w, w->prec, w->recon, 0);
  b.in = w->t;
  b.in_fb = w->fb;
  b.out = w->r;
  b.out_fb = w->fb;
  b.p = w->p;
  b.p_fb = w->fb;
  b.xs = w->xs;
  b.xs_fb = w->xs_fb;
  b.xs_prec = xs_prec(w->prec);
  b.partial = w->partial + w->partial_stride;
  b.counter = w->counters + w->counter_stride;
  b.gate = GATE_RUNNING;
  rc = check_launch(w->ctx, launch_dslash(w->prec, w->recon, w->cfg_update.nr, MODE_UPDATE,
                                          w->prec, b, w->cfg_update.block, st));
  if (rc) return rc;
  {
    VecArgs f = vec_args(w, 1);
    f.checkpoint = checkpoint;
    if ((rc = check_launch(w->ctx, launch_cg_finish(1, f, st)))) return rc;
  }
  if (checkpoint && (rc = cg_enqueue_ru(w, st))) return rc;
  return cg_enqueue_xpay(w, st);
}

int cg_enqueue_block(CGWork *w, int k, bool graph, cudaStream_t st) {
  // reliable updates can follow every RU_PERIOD-th iteration of a block
  if (!graph) {
    for (int it = 0; it < k; ++it) {
      int rc = cg_enqueue_iteration(w, st, (it + 1) % RU_PERIOD == 0);
      if (rc) return rc;
    }
    return SQ_OK;
  }
  if (!w->exec || w->exec_iters != k) {
    if (w->exec) {
      cudaGraphExecDestroy(w->exec);
      w->exec = nullptr;
    }
    uint64_t before = w->ctx->launches.load();
    cudaGraph_t g = nullptr;
    SQ_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = SQ_OK;
    for (int it = 0; it < k && rc == SQ_OK; ++it)
      rc = cg_enqueue_iteration(w, st, (it + 1) % RU_PERIOD == 0);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    w->exec_kernels = (int)(w->ctx->launches.load() - before);
    w->ctx->launches = before;  // counted on replay
    if (rc != SQ_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      return rc;
    }
    SQ_CUDA_TRY(e);
    e = cudaGraphInstantiate(&w->exec, g, 0);
    cudaGraphDestroy(g);
    SQ_CUDA_TRY(e);
    w->exec_iters = k;
  }
  SQ_CUDA_TRY(cudaGraphLaunch(w->exec, st));
  w->ctx->launches += w->exec_kernels;
  return SQ_OK;
}

static bool any_running(const CGWork *w) {
  for (int k = 0; k < w->nrhs; ++k)
    if (cg_slot_live(w->slots_h[k].status)) return true;
  return false;
}

int cg_run(CGWork *w, int block_iters, bool graph, cudaStream_t st) {
  int rc;
  // whole checkpoint periods per block
  block_iters = (block_iters + RU_PERIOD - 1) / RU_PERIOD * RU_PERIOD;
  if ((rc = cg_slots_download(w, st))) return rc;
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  while (any_running(w)) {
    if ((rc = cg_enqueue_block(w, block_iters, graph, st))) return rc;
    if ((rc = cg_slots_download(w, st))) return rc;
    SQ_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return SQ_OK;
}

int slot_status_to_sq(int s) {
  switch (s) {
    case SLOT_CONVERGED: return SQ_OK;
    case SLOT_MAXITER: return SQ_NOT_CONVERGED;
    case SLOT_NONFINITE: return SQ_ERR_NONFINITE;
    case SLOT_RUNNING:
    case SLOT_WAIT:
    case SLOT_INIT: return SQ_PENDING;
    default: return SQ_ERR_ARG;
  }
}

void fill_launch_stats(const CGWork *w, sq_cg_stats *st) {
  if (!st) return;
  st->oe_block = std::min(w->cfg_norm.block, dslash_max_block(w->prec, w->cfg_norm.nr));
  st->oe_rhs_tile = w->cfg_norm.nr;
  st->eo_block = std::min(w->cfg_update.block, dslash_max_block(w->prec, w->cfg_update.nr));
  st->eo_rhs_tile = w->cfg_update.nr;
}

void fill_stats(const SlotState &s, double seconds, long vh, sq_cg_stats *st) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->status = slot_status_to_sq(s.status);
  st->iterations = s.iter;
  st->reliable_updates = s.n_ru;
  st->true_residual = (s.b2 > 0) ? std::sqrt(s.rr_true / s.b2) : 0.0;
  st->seconds = seconds;
  st->gflops = (seconds > 0) ? 2364.0 * (double)vh * s.iter / seconds * 1e-9 : 0.0;
}

}  // namespace sq
