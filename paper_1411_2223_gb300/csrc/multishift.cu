// Multi-shift CG on the GPU: (m_i^2 - D_eo D_oe) x_i = b for all masses from
// the Krylov space of the smallest mass (Jegerlehner's shifted recurrences),
// in the sloppy precision, followed by a batched mixed-precision refinement
// of every shift started from its shifted solution.
//
// One iteration = four kernels: the base system's two Dslash (the second one
// also yields alpha and the shifted alpha_i), ms_update (r -= alpha Ap,
// |r|^2; beta, beta_i, per-shift convergence) and ms_xpay (x_i += alpha_i p_i,
// p_i = zeta_i r + beta_i p_i for every shift).
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "cg_finish.cuh"
#include "sq_device.cuh"
#include "sq_host.h"

namespace sq {

namespace {

struct MsArgs {
  Geom g;
  int nshift, base;
  char *r, *ap, *p, *x;     // r, Ap: 1 field; p, x: nshift fields
  size_t fb, xfb;
  const char *b64;
  SlotState *bs;
  ShiftState *sh;
  double *partial;
  unsigned *counter;
};

__device__ __forceinline__ bool ms_live(const SlotState *b) {
  return b->status == SLOT_RUNNING || b->status == SLOT_WAIT;
}

template <int S>
__global__ void __launch_bounds__(256) ms_init_kernel(MsArgs a) {
  using R = typename SpinorIO<S>::R;
  constexpr int XP = (S == PREC_F64) ? PREC_F64 : PREC_F32;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int St = a.g.stride;
  double val[1] = {0.0};
  if (i < a.g.vh) {
    Vec3<double> b = SpinorIO<PREC_F64>::load(a.b64, St, i);
    double n2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) n2 = fma(b.c[c].x, b.c[c].x, fma(b.c[c].y, b.c[c].y, n2));
    val[0] = n2;
    Vec3<R> rv = convert<R>(b);
    SpinorIO<S>::store(a.r, St, i, rv);
    Vec3<typename SpinorIO<XP>::R> z;
    zero(z);
    for (int k = 0; k < a.nshift; ++k) {
      SpinorIO<S>::store(a.p + k * a.fb, St, i, rv);
      SpinorIO<XP>::store(a.x + k * a.xfb, St, i, z);
    }
  }
  double *const inst[1] = {a.partial};
  double sum[1];
  if (warp_tree_reduce<1>(val, 1, inst, a.g, i, a.counter, sum)) {
    if ((threadIdx.x & 31) == 0) {
      const double b2 = sum[0];
      finish_init(a.bs, b2);
      a.bs->alpha_prev = 1.0;
      a.bs->beta_prev = 0.0;
      for (int k = 0; k < a.nshift; ++k) {
        ShiftState &s = a.sh[k];
        s.zeta = s.zeta_prev = s.zeta_next = 1.0;
        s.alpha = s.beta = 0.0;
        s.tol2b2 = a.bs->tol2b2;
        s.active = s.cont = (a.bs->status == SLOT_RUNNING);
        s.iter = 0;
      }
    }
  }
}

// r -= alpha Ap ; |r|^2 ; last block: finish_shift_update
template <int S>
__global__ void __launch_bounds__(256) ms_update_kernel(MsArgs a) {
  using R = typename SpinorIO<S>::R;
  if (a.bs->status != SLOT_RUNNING) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int St = a.g.stride;
  double val[1] = {0.0};
  if (i < a.g.vh) {
    const R al = (R)a.bs->alpha;
    Vec3<R> ap = SpinorIO<S>::load(a.ap, St, i);
    Vec3<R> rv = SpinorIO<S>::load(a.r, St, i);
    R n2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rv.c[c].x = fma(-al, ap.c[c].x, rv.c[c].x);
      rv.c[c].y = fma(-al, ap.c[c].y, rv.c[c].y);
      n2 = fma(rv.c[c].x, rv.c[c].x, fma(rv.c[c].y, rv.c[c].y, n2));
    }
    SpinorIO<S>::store(a.r, St, i, rv);
    val[0] = (double)n2;
  }
  double *const inst[1] = {a.partial};
  double rr[1];
  if (warp_tree_reduce<1>(val, 1, inst, a.g, i, a.counter, rr) && (threadIdx.x & 31) == 0)
    finish_shift_update(a.bs, a.sh, a.nshift, rr[0]);
}

// x_i += alpha_i p_i ; p_i = zeta_i r + beta_i p_i ; the last block closes
// the iteration (active <- cont, and a waiting base takes its final status).
template <int S>
__global__ void __launch_bounds__(256) ms_xpay_kernel(MsArgs a) {
  using R = typename SpinorIO<S>::R;
  constexpr int XP = (S == PREC_F64) ? PREC_F64 : PREC_F32;
  if (!ms_live(a.bs)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int St = a.g.stride;
  if (i < a.g.vh) {
    Vec3<R> rv = SpinorIO<S>::load(a.r, St, i);
    const bool base_cont = a.bs->status == SLOT_RUNNING;
    for (int k = 0; k < a.nshift; ++k) {
      const ShiftState &s = a.sh[k];
      const bool pc = (k == a.base) ? base_cont : (s.cont != 0 && base_cont);
      if (!s.active && !pc) continue;
      Vec3<R> p = SpinorIO<S>::load(a.p + k * a.fb, St, i);
      if (s.active) {
        const R al = (R)s.alpha;
        auto x = SpinorIO<XP>::load(a.x + k * a.xfb, St, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x.c[c].x = fma(al, p.c[c].x, x.c[c].x);
          x.c[c].y = fma(al, p.c[c].y, x.c[c].y);
        }
        SpinorIO<XP>::store(a.x + k * a.xfb, St, i, x);
      }
      if (pc) {
        const R z = (R)s.zeta, be = (R)s.beta;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          p.c[c].x = fma(z, rv.c[c].x, be * p.c[c].x);
          p.c[c].y = fma(z, rv.c[c].y, be * p.c[c].y);
        }
        SpinorIO<S>::store(a.p + k * a.fb, St, i, p);
      }
    }
  }
  unsigned *close = a.counter + ticket_stride(a.g);
  if (last_block_arrived(close, gridDim.x)) {
    if (threadIdx.x == 0) {
      for (int k = 0; k < a.nshift; ++k) a.sh[k].active = a.sh[k].cont;
      if (a.bs->status == SLOT_WAIT) a.bs->status = a.bs->final_status;
      *close = 0;
    }
  }
}

template <template <int> class K, typename... Args>
int launch_prec(int prec, dim3 grid, cudaStream_t st, Args... args) {
  switch (prec) {
    case PREC_F64: K<PREC_F64>::run(grid, st, args...); return 0;
    case PREC_F32: K<PREC_F32>::run(grid, st, args...); return 0;
    case PREC_I16: K<PREC_I16>::run(grid, st, args...); return 0;
  }
  return -1;
}

template <int S> struct InitL {
  static void run(dim3 g, cudaStream_t st, const MsArgs &a) { ms_init_kernel<S><<<g, 256, 0, st>>>(a); }
};
template <int S> struct UpdL {
  static void run(dim3 g, cudaStream_t st, const MsArgs &a) { ms_update_kernel<S><<<g, 256, 0, st>>>(a); }
};
template <int S> struct XpayL {
  static void run(dim3 g, cudaStream_t st, const MsArgs &a) { ms_xpay_kernel<S><<<g, 256, 0, st>>>(a); }
};

// Workspace of one multi-shift solve shape (cached per context).
struct MsWork {
  sq_ctx *ctx = nullptr;
  GaugeField *gf = nullptr;
  int prec = PREC_F32, recon = 18, nshift = 0, base = 0;
  size_t fb = 0, xfb = 0, f64_fb = 0, bytes = 0;
  char *b64 = nullptr, *r = nullptr, *ap = nullptr, *t = nullptr, *p = nullptr, *x = nullptr;
  double *canon = nullptr;  // 2 * nshift canonical vectors: sources, solutions
  SlotState *bs_d = nullptr, *bs_h = nullptr;
  ShiftState *sh_d = nullptr, *sh_h = nullptr;
  double *partial = nullptr;
  unsigned *counters = nullptr;
  cudaGraphExec_t exec = nullptr;
  int exec_iters = 0, exec_kernels = 0;
  DslashConfig cfg, cfg_mdagm;

  ~MsWork() {
    if (exec) cudaGraphExecDestroy(exec);
    if (bs_h) cudaFreeHost(bs_h);
    if (sh_h) cudaFreeHost(sh_h);
    void *bufs[] = {b64, r, ap, t, p, x, canon, bs_d, sh_d, partial, counters};
    for (void *b : bufs)
      if (b) cudaFree(b);
    if (ctx) {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->in_use -= bytes;
    }
    if (gf) gf->users--;
  }
};

std::mutex g_ms_mu;
std::map<std::tuple<const sq_ctx *, int, int, int, int>, std::unique_ptr<MsWork>> g_ms;

int ms_work_get(sq_ctx *ctx, GaugeField *gf, int gid, int prec, int recon, int nshift,
                MsWork **out) {
  std::lock_guard<std::mutex> lk(g_ms_mu);
  auto key = std::make_tuple((const sq_ctx *)ctx, gid, prec, recon, nshift);
  auto it = g_ms.find(key);
  if (it != g_ms.end()) {
    *out = it->second.get();
    return SQ_OK;
  }
  std::unique_ptr<MsWork> w(new MsWork());
  const Geom &g = gf->g;
  w->gf = gf;
  gf->users++;
  w->prec = prec;
  w->recon = recon;
  w->nshift = nshift;
  w->fb = spinor_bytes(prec, g.stride);
  w->xfb = spinor_bytes(xs_prec(prec), g.stride);
  w->f64_fb = spinor_bytes(PREC_F64, g.stride);
  const size_t canon_b = (size_t)3 * g.vh * 16;
  size_t sizes[] = {w->f64_fb, w->fb, w->fb, w->fb, w->fb * nshift, w->xfb * nshift,
                    2 * canon_b * nshift, sizeof(SlotState), sizeof(ShiftState) * nshift,
                    sizeof(double) * red_stride(g), sizeof(unsigned) * (2 * ticket_stride(g) + 4)};
  char **ptrs[] = {&w->b64, &w->r, &w->ap, &w->t, &w->p, &w->x};
  size_t total = 0;
  for (size_t s : sizes) total += s;
  {
    std::lock_guard<std::mutex> l2(ctx->mu);
    if (ctx->in_use + total > ctx->budget) return SQ_ERR_OOM;
    ctx->in_use += total;
  }
  w->ctx = ctx;
  w->bytes = total;
  for (int k = 0; k < 6; ++k) {
    SQ_CUDA_TRY(cudaMalloc((void **)ptrs[k], sizes[k]));
    SQ_CUDA_TRY(cudaMemset(*ptrs[k], 0, sizes[k]));
  }
  SQ_CUDA_TRY(cudaMalloc((void **)&w->canon, sizes[6]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->bs_d, sizes[7]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->sh_d, sizes[8]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->partial, sizes[9]));
  SQ_CUDA_TRY(cudaMalloc((void **)&w->counters, sizes[10]));
  SQ_CUDA_TRY(cudaMemset(w->counters, 0, sizes[10]));
  SQ_CUDA_TRY(cudaMallocHost((void **)&w->bs_h, sizes[7]));
  SQ_CUDA_TRY(cudaMallocHost((void **)&w->sh_h, sizes[8]));
  *out = w.get();
  g_ms[key] = std::move(w);
  return SQ_OK;
}

MsArgs ms_args(MsWork *w) {
  MsArgs a;
  a.g = w->gf->g;
  a.nshift = w->nshift;
  a.base = w->base;
  a.r = w->r;
  a.ap = w->ap;
  a.p = w->p;
  a.x = w->x;
  a.fb = w->fb;
  a.xfb = w->xfb;
  a.b64 = w->b64;
  a.bs = w->bs_d;
  a.sh = w->sh_d;
  a.partial = w->partial;
  a.counter = w->counters;
  return a;
}

int ms_enqueue_iteration(MsWork *w, cudaStream_t st) {
  sq_ctx *ctx = w->ctx;
  const Geom &g = w->gf->g;
  const char *pb = w->p + (size_t)w->base * w->fb;
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.nrhs = 1;
  a.slots = w->bs_d;
  a.gate = GATE_RUNNING;
  a.out_parity = 1;
  a.links = w->gf->link_ptr(w->prec, w->recon, 1);
  a.ls = w->gf->scales(w->prec, w->recon);
  a.in = pb;
  a.out = w->t;
  if (launch_dslash(w->prec, w->recon, 1, MODE_PLAIN, w->prec, a, w->cfg.block, st)) return SQ_ERR_ARG;
  DslashArgs b = a;
  b.out_parity = 0;
  b.links = w->gf->link_ptr(w->prec, w->recon, 0);
  b.in = w->t;
  b.out = w->ap;
  b.p = pb;
  b.partial = w->partial;
  b.counter = w->counters + ticket_stride(g) + 1;
  b.shifts = w->sh_d;
  b.nshift = w->nshift;
  if (launch_dslash(w->prec, w->recon, 1, MODE_MDAGM, w->prec, b, w->cfg_mdagm.block, st))
    return SQ_ERR_ARG;
  dim3 grid((g.vh + 255) / 256);
  MsArgs m = ms_args(w);
  if (launch_prec<UpdL>(w->prec, grid, st, m)) return SQ_ERR_ARG;
  if (launch_prec<XpayL>(w->prec, grid, st, m)) return SQ_ERR_ARG;
  ctx->launches += 4;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "multi-shift launch", __FILE__, __LINE__);
    return SQ_ERR_CUDA;
  }
  return SQ_OK;
}

int ms_enqueue_block(MsWork *w, int k, bool graph, cudaStream_t st) {
  if (!graph) {
    for (int it = 0; it < k; ++it) {
      int rc = ms_enqueue_iteration(w, st);
      if (rc) return rc;
    }
    return SQ_OK;
  }
  if (!w->exec || w->exec_iters != k) {
    if (w->exec) cudaGraphExecDestroy(w->exec);
    w->exec = nullptr;
    uint64_t before = w->ctx->launches.load();
    cudaGraph_t gr;
    SQ_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = SQ_OK;
    for (int it = 0; it < k && rc == SQ_OK; ++it) rc = ms_enqueue_iteration(w, st);
    cudaError_t e = cudaStreamEndCapture(st, &gr);
    w->exec_kernels = (int)(w->ctx->launches.load() - before);
    w->ctx->launches = before;
    if (rc) {
      if (e == cudaSuccess) cudaGraphDestroy(gr);
      return rc;
    }
    SQ_CUDA_TRY(e);
    e = cudaGraphInstantiate(&w->exec, gr, 0);
    cudaGraphDestroy(gr);
    SQ_CUDA_TRY(e);
    w->exec_iters = k;
  }
  SQ_CUDA_TRY(cudaGraphLaunch(w->exec, st));
  w->ctx->launches += w->exec_kernels;
  return SQ_OK;
}

}  // namespace

void drop_multishift_works(const sq_ctx *ctx, int gid) {
  std::lock_guard<std::mutex> lk(g_ms_mu);
  for (auto it = g_ms.begin(); it != g_ms.end();) {
    if (std::get<0>(it->first) == ctx && (gid < 0 || std::get<1>(it->first) == gid))
      it = g_ms.erase(it);
    else
      ++it;
  }
}

int solve_batch_locked(sq_ctx *ctx, int gauge_id, int nrhs, const double *src,
                       const double *masses, double tol, const sq_cg_opts *opts_in, double *x,
                       sq_cg_stats *stats);

}  // namespace sq

using namespace sq;

extern "C" int cg_solve_multishift(sq_ctx *ctx, int gauge_id, const double *src, int nshift,
                                   const double *masses, double tol, const sq_cg_opts *opts_in,
                                   double *x, sq_cg_stats *stats) {
  if (!ctx || !src || !masses || !x || nshift < 1 || nshift > 16) return SQ_ERR_ARG;
  if (!(tol > 0) || !std::isfinite(tol)) return SQ_ERR_ARG;
  for (int k = 0; k < nshift; ++k)
    if (!(masses[k] > 0) || !std::isfinite(masses[k])) return SQ_ERR_ARG;
  sq_cg_opts o;
  sq_cg_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (o.precision < 0 || o.precision > 2 || (o.long_recon != 18 && o.long_recon != 12))
    return SQ_ERR_ARG;
  if (o.max_iter < 1 || o.block_iters < 1) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(o.precision, o.long_recon) || !gf->has(PREC_F64, 18)) return SQ_ERR_UNSUPPORTED;
  const bool dev = (o.flags & SQ_CG_DEVICE_PTRS) != 0;
  const size_t vec = (size_t)3 * gf->g.vh;  // complex per vector
  if (!dev)
    for (size_t k = 0; k < 2 * vec; ++k)
      if (!std::isfinite(src[k])) return SQ_ERR_NONFINITE;

  std::lock_guard<std::mutex> solve_lock(ctx->solve_mu);
  cudaSetDevice(ctx->device);
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = ctx->stream;
  cudaStream_t user = (cudaStream_t)o.stream;
  if (user == cudaStreamLegacy || user == cudaStreamPerThread) user = nullptr;
  if (user) st = user;
  else  // a default stream (NULL: the legacy one): the caller's work on it first
    SQ_CUDA_TRY(cudaStreamSynchronize(o.stream ? (cudaStream_t)o.stream : cudaStreamLegacy));

  MsWork *w = nullptr;
  int rc = ms_work_get(ctx, gf, gauge_id, o.precision, o.long_recon, nshift, &w);
  if (rc) return rc;
  int base = 0;
  for (int k = 1; k < nshift; ++k)
    if (masses[k] < masses[base]) base = k;
  if (w->exec && w->base != base) {
    cudaGraphExecDestroy(w->exec);
    w->exec = nullptr;
  }
  w->base = base;
  w->cfg = tuned_dslash(ctx, *gf, o.precision, o.long_recon, 1, MODE_PLAIN, st);
  w->cfg_mdagm = tuned_dslash(ctx, *gf, o.precision, o.long_recon, 1, MODE_MDAGM, st);

  // sources: nshift canonical copies of b (device); solutions follow them
  double *csrc = w->canon, *cx = w->canon + 2 * vec * nshift;
  const size_t vb = vec * 16;
  SQ_CUDA_TRY(cudaMemcpyAsync(csrc, src, vb, dev ? cudaMemcpyDeviceToDevice
                                                 : cudaMemcpyHostToDevice, st));
  for (int k = 1; k < nshift; ++k)
    SQ_CUDA_TRY(cudaMemcpyAsync(csrc + 2 * vec * k, csrc, vb, cudaMemcpyDeviceToDevice, st));
  if (launch_pack(PREC_F64, gf->g, csrc, vec, w->b64, w->f64_fb, 1, st)) return SQ_ERR_ARG;
  ctx->launches++;

  // sloppy tolerance of the shifted phase; the refinement reaches tol.  An
  // FP32 shifted iteration moves the base system's two Dslash and each
  // shift's x and p (about 3.3 KB per site for 8 shifts), a refinement
  // iteration two Dslash per shift: 8 masses at 24^3 x 64 to 1e-8 took
  // 167.5 ms with 1e-5 here, 161.4 ms with 1e-6 and 163.0 ms with 1e-7.
  const double tol_ms = std::max(tol, o.precision == PREC_F64 ? tol
                                     : o.precision == PREC_F32 ? 1e-6 : 1e-3);
  std::memset(w->bs_h, 0, sizeof(SlotState));
  w->bs_h->m2 = masses[base] * masses[base];
  w->bs_h->tol2 = tol_ms * tol_ms;
  w->bs_h->max_iter = o.max_iter;
  w->bs_h->status = SLOT_RUNNING;
  for (int k = 0; k < nshift; ++k) {
    std::memset(&w->sh_h[k], 0, sizeof(ShiftState));
    w->sh_h[k].sigma = masses[k] * masses[k] - masses[base] * masses[base];
  }
  SQ_CUDA_TRY(cudaMemcpyAsync(w->bs_d, w->bs_h, sizeof(SlotState), cudaMemcpyHostToDevice, st));
  SQ_CUDA_TRY(cudaMemcpyAsync(w->sh_d, w->sh_h, sizeof(ShiftState) * nshift,
                              cudaMemcpyHostToDevice, st));
  MsArgs m = ms_args(w);
  if (launch_prec<InitL>(o.precision, dim3((gf->g.vh + 255) / 256), st, m)) return SQ_ERR_ARG;
  ctx->launches++;
  const bool graph = !(o.flags & SQ_CG_NO_GRAPH);
  for (;;) {
    SQ_CUDA_TRY(cudaMemcpyAsync(w->bs_h, w->bs_d, sizeof(SlotState), cudaMemcpyDeviceToHost, st));
    SQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (w->bs_h->status != SLOT_RUNNING && w->bs_h->status != SLOT_WAIT) break;
    if ((rc = ms_enqueue_block(w, o.block_iters, graph, st))) return rc;
  }
  SQ_CUDA_TRY(cudaMemcpyAsync(w->sh_h, w->sh_d, sizeof(ShiftState) * nshift,
                              cudaMemcpyDeviceToHost, st));
  const int ms_status = w->bs_h->status;
  // shifted solutions -> canonical FP64 initial guesses
  if (launch_unpack(xs_prec(o.precision), gf->g, w->x, w->xfb, cx, vec, nshift, st))
    return SQ_ERR_ARG;
  ctx->launches++;
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  if (ms_status == SLOT_NONFINITE) return SQ_ERR_NONFINITE;

  // refinement: batched mixed-precision CG from the shifted solutions
  sq_cg_opts ro = o;
  ro.flags = SQ_CG_DEVICE_PTRS | SQ_CG_INITIAL_GUESS | (o.flags & SQ_CG_NO_GRAPH);
  ro.stream = (void *)st;
  std::vector<sq_cg_stats> rs(nshift);
  rc = solve_batch_locked(ctx, gauge_id, nshift, csrc, masses, tol, &ro, cx, rs.data());
  if (rc < 0) return rc;
  const size_t out_b = vb * nshift;
  if (dev) SQ_CUDA_TRY(cudaMemcpyAsync(x, cx, out_b, cudaMemcpyDeviceToDevice, st));
  else SQ_CUDA_TRY(cudaMemcpyAsync(x, cx, out_b, cudaMemcpyDeviceToHost, st));
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int k = 0; k < nshift; ++k) {
      stats[k] = rs[k];
      stats[k].iterations += w->sh_h[k].iter;
      stats[k].seconds = secs;
      stats[k].gflops = secs > 0 ? 2364.0 * gf->g.vh * stats[k].iterations / secs * 1e-9 : 0;
    }
  return rc;
}
