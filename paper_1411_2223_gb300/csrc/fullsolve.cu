// Full-lattice staggered solve and the unpreconditioned operator.
//
// The staggered Dirac matrix M = m + D couples only sites of opposite parity,
//   M = [ m     D_eo ]
//       [ D_oe  m    ],
// so M x = b reduces to the even-site system the CG solves,
//   (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o,
// followed by the odd sites from the second row,
//   x_o = (b_o - D_oe x_e) / m.
// The even residual r~ = m b_e - D_eo b_o - A x_e and the full one satisfy
// b - M x = (r~ / m, 0), so the even system is solved to
// tol * m |b| / |m b_e - D_eo b_o| to give |b - M x| / |b| <= tol.  The paper's
// CG inverter (Sec. 2, Fig. 1) solves the staggered equation on the whole
// lattice; this file is the step from the even-site CG to that solution.
// Everything here runs in FP64 on the device; the full residual is
// recomputed with two FP64 Dslash applications after the solve.
#include <chrono>
#include <cmath>
#include <cstring>

#include "sq_host.h"

namespace sq {

int solve_batch_locked(sq_ctx *ctx, int gauge_id, int nrhs, const double *src,
                       const double *masses, double tol, const sq_cg_opts *opts_in, double *x,
                       sq_cg_stats *stats);

namespace {

// canonical full-lattice [site_lex][colour] complex128 -> packed FP64 half of `parity`
__global__ void full_to_half_kernel(Geom g, int parity, const double2 *full, char *half) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  const SiteCoords s = site_coords(g, parity, i);
  const double2 *c = full + (size_t)3 * s.lex;
  Vec3<double> v;
#pragma unroll
  for (int k = 0; k < 3; ++k) v.c[k] = c[k];
  SpinorIO<PREC_F64>::store(half, g.stride, i, v);
}

__global__ void half_to_full_kernel(Geom g, int parity, const char *half, double2 *full) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  const SiteCoords s = site_coords(g, parity, i);
  const Vec3<double> v = SpinorIO<PREC_F64>::load(half, g.stride, i);
  double2 *c = full + (size_t)3 * s.lex;
#pragma unroll
  for (int k = 0; k < 3; ++k) c[k] = v.c[k];
}

// out = a x + b y + c z on packed FP64 halves (z may be null)
__global__ void lincomb_kernel(Geom g, double a, const char *x, double b, const char *y, double c,
                               const char *z, char *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  const Vec3<double> vx = SpinorIO<PREC_F64>::load(x, g.stride, i);
  const Vec3<double> vy = SpinorIO<PREC_F64>::load(y, g.stride, i);
  Vec3<double> o;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    o.c[k].x = fma(a, vx.c[k].x, b * vy.c[k].x);
    o.c[k].y = fma(a, vx.c[k].y, b * vy.c[k].y);
  }
  if (z != nullptr) {
    const Vec3<double> vz = SpinorIO<PREC_F64>::load(z, g.stride, i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o.c[k].x = fma(c, vz.c[k].x, o.c[k].x);
      o.c[k].y = fma(c, vz.c[k].y, o.c[k].y);
    }
  }
  SpinorIO<PREC_F64>::store(out, g.stride, i, o);
}

// |v|^2 of a packed FP64 half: fixed 128-site chunk partials, then one block
// adds them in a fixed order (the same bits for every launch shape).
constexpr int FS_BLOCK = 256;

__global__ void norm2_partial_kernel(Geom g, const char *v, double *partial) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double val[1] = {0.0};
  if (i < g.vh) {
    const Vec3<double> a = SpinorIO<PREC_F64>::load(v, g.stride, i);
#pragma unroll
    for (int k = 0; k < 3; ++k) val[0] = fma(a.c[k].x, a.c[k].x, fma(a.c[k].y, a.c[k].y, val[0]));
  }
  __shared__ double smem[FS_BLOCK / 32];
  chunk_reduce<1>(val, smem, partial, g.nchunks);
}

__global__ void sum_partials_kernel(const double *partial, int n, double *out) {
  __shared__ double red[32];
  const double s = block_sum_fixed(partial, n, red);
  if (threadIdx.x == 0) *out = s;
}

inline unsigned blocks(const Geom &g) { return (unsigned)((g.vh + FS_BLOCK - 1) / FS_BLOCK); }

// Device scratch of one full-lattice operation (released on destruction).
struct FullWork {
  sq_ctx *ctx = nullptr;
  void *base = nullptr;
  size_t bytes = 0;
  ~FullWork() {
    if (base) ctx->release(base, bytes);
  }
};

struct FullOps {
  sq_ctx *ctx;
  GaugeField *gf;
  cudaStream_t st;
  DslashConfig cfg;

  int dslash(int out_parity, const char *in, char *out) {
    DslashArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = gf->g;
    a.out_parity = out_parity;
    a.links = gf->link_ptr(PREC_F64, 18, out_parity);
    a.ls = gf->scales(PREC_F64, 18);
    a.in = in;
    a.out = out;
    a.in_fb = a.out_fb = spinor_bytes(PREC_F64, gf->g.stride);
    a.nrhs = 1;
    a.gate = GATE_NONE;
    if (launch_dslash(PREC_F64, 18, 1, MODE_PLAIN, PREC_F64, a, cfg.block, st)) return SQ_ERR_ARG;
    ctx->launches++;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
  int lincomb(double a, const char *x, double b, const char *y, double c, const char *z,
              char *out) {
    if (gf->g.vh <= 0) return SQ_OK;
    lincomb_kernel<<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, a, x, b, y, c, z, out);
    ctx->launches++;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
  int split(const double *full, char *even, char *odd) {
    const double2 *f = reinterpret_cast<const double2 *>(full);
    full_to_half_kernel<<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, 0, f, even);
    full_to_half_kernel<<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, 1, f, odd);
    ctx->launches += 2;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
  int merge(const char *even, const char *odd, double *full) {
    double2 *f = reinterpret_cast<double2 *>(full);
    half_to_full_kernel<<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, 0, even, f);
    half_to_full_kernel<<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, 1, odd, f);
    ctx->launches += 2;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
  // *out (device double) = |v|^2
  int norm2(const char *v, double *partial, double *out) {
    norm2_partial_kernel<<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, v, partial);
    sum_partials_kernel<<<1, 128, 0, st>>>(partial, gf->g.nchunks, out);
    ctx->launches += 2;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
};

cudaStream_t pick_stream(sq_ctx *ctx, void *user_stream) {
  cudaStream_t user = (cudaStream_t)user_stream;
  if (user == cudaStreamLegacy || user == cudaStreamPerThread) user = nullptr;
  return user ? user : ctx->stream;
}

bool all_finite(const double *p, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

}  // namespace
}  // namespace sq

using namespace sq;

extern "C" int dirac_apply(sq_ctx *ctx, int gauge_id, double mass, const double *in_dev,
                           double *out_dev, void *stream) {
  if (!ctx || !in_dev || !out_dev || in_dev == out_dev || !std::isfinite(mass)) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(PREC_F64, 18)) return SQ_ERR_UNSUPPORTED;
  cudaSetDevice(ctx->device);
  const Geom &g = gf->g;
  cudaStream_t st = pick_stream(ctx, stream);
  if (st == ctx->stream && stream) SQ_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  const size_t fb = spinor_bytes(PREC_F64, g.stride);
  FullWork w;
  w.ctx = ctx;
  w.bytes = 4 * fb;
  int rc = ctx->alloc(w.bytes, &w.base);
  if (rc) return rc;
  char *ie = static_cast<char *>(w.base), *io = ie + fb, *oe = io + fb, *oo = oe + fb;
  FullOps ops{ctx, gf, st, tuned_dslash(ctx, *gf, PREC_F64, 18, 1, MODE_PLAIN, st)};
  if ((rc = ops.split(in_dev, ie, io))) return rc;
  // out_e = m in_e + D_eo in_o, out_o = m in_o + D_oe in_e
  if ((rc = ops.dslash(0, io, oe))) return rc;
  if ((rc = ops.dslash(1, ie, oo))) return rc;
  if ((rc = ops.lincomb(mass, ie, 1.0, oe, 0.0, nullptr, oe))) return rc;
  if ((rc = ops.lincomb(mass, io, 1.0, oo, 0.0, nullptr, oo))) return rc;
  if ((rc = ops.merge(oe, oo, out_dev))) return rc;
  // the scratch is released on return: finish before that
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  return SQ_OK;
}

extern "C" int cg_solve_full(sq_ctx *ctx, int gauge_id, const double *src, double mass,
                             double tol, const sq_cg_opts *opts_in, double *x,
                             sq_cg_stats *stats) {
  if (!ctx || !src || !x) return SQ_ERR_ARG;
  if (!(mass > 0) || !std::isfinite(mass) || !(tol > 0) || !std::isfinite(tol)) return SQ_ERR_ARG;
  sq_cg_opts o;
  sq_cg_opts_default(&o);
  if (opts_in) o = *opts_in;
  std::lock_guard<std::mutex> solve_lock(ctx->solve_mu);
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(PREC_F64, 18)) return SQ_ERR_UNSUPPORTED;
  const Geom &g = gf->g;
  const bool dev = (o.flags & SQ_CG_DEVICE_PTRS) != 0;
  const bool guess = (o.flags & SQ_CG_INITIAL_GUESS) != 0;
  const size_t vol = (size_t)2 * g.vh;
  const size_t full_bytes = vol * 3 * 16, half_canon = (size_t)g.vh * 3 * 16;
  if (!dev && !all_finite(src, vol * 6)) return SQ_ERR_NONFINITE;
  cudaSetDevice(ctx->device);
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = pick_stream(ctx, o.stream);
  if (st == ctx->stream && o.stream) SQ_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)o.stream));

  const size_t fb = spinor_bytes(PREC_F64, g.stride);
  FullWork w;
  w.ctx = ctx;
  const size_t nparts = (size_t)g.nchunks;
  w.bytes = 7 * fb + 2 * half_canon + (dev ? 0 : full_bytes) + (nparts + 8) * sizeof(double);
  int rc = ctx->alloc(w.bytes, &w.base);
  if (rc) return rc;
  char *p = static_cast<char *>(w.base);
  char *be = p, *bo = be + fb, *xe = bo + fb, *xo = xe + fb, *t = xo + fb, *re = t + fb,
       *ro = re + fb;
  double *bt_c = reinterpret_cast<double *>(ro + fb);
  double *xe_c = reinterpret_cast<double *>(reinterpret_cast<char *>(bt_c) + half_canon);
  char *after = reinterpret_cast<char *>(xe_c) + half_canon;
  double *stage = dev ? nullptr : reinterpret_cast<double *>(after);
  double *partial = reinterpret_cast<double *>(after + (dev ? 0 : full_bytes));
  double *sums = partial + nparts;  // |b_e|^2, |b_o|^2, |b~|^2, |r_e|^2, |r_o|^2
  FullOps ops{ctx, gf, st, tuned_dslash(ctx, *gf, PREC_F64, 18, 1, MODE_PLAIN, st)};

  const double *bsrc = src;
  if (!dev) {
    SQ_CUDA_TRY(cudaMemcpyAsync(stage, src, full_bytes, cudaMemcpyHostToDevice, st));
    bsrc = stage;
  }
  if ((rc = ops.split(bsrc, be, bo))) return rc;
  // b~ = m b_e - D_eo b_o
  if ((rc = ops.dslash(0, bo, t))) return rc;
  if ((rc = ops.lincomb(mass, be, -1.0, t, 0.0, nullptr, re))) return rc;
  if ((rc = ops.norm2(be, partial, sums + 0))) return rc;
  if ((rc = ops.norm2(bo, partial, sums + 1))) return rc;
  if ((rc = ops.norm2(re, partial, sums + 2))) return rc;
  if (launch_unpack(PREC_F64, g, re, fb, bt_c, (size_t)3 * g.vh, 1, st)) return SQ_ERR_ARG;
  ctx->launches++;
  double h[3];
  SQ_CUDA_TRY(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  const double b2 = h[0] + h[1], bt2 = h[2];
  if (!std::isfinite(b2) || !std::isfinite(bt2)) return SQ_ERR_NONFINITE;

  sq_cg_stats est;
  std::memset(&est, 0, sizeof(est));
  int status = SQ_OK;
  if (guess) {  // even half of the caller's guess starts the even-site CG
    const double *gsrc = x;
    if (!dev) {
      if (!all_finite(x, vol * 6)) return SQ_ERR_NONFINITE;
      SQ_CUDA_TRY(cudaMemcpyAsync(stage, x, full_bytes, cudaMemcpyHostToDevice, st));
      gsrc = stage;
    }
    if ((rc = ops.split(gsrc, xe, xo))) return rc;
    if (launch_unpack(PREC_F64, g, xe, fb, xe_c, (size_t)3 * g.vh, 1, st)) return SQ_ERR_ARG;
    ctx->launches++;
  }
  if (b2 == 0.0 || bt2 == 0.0) {
    // b~ = 0: x_e = 0 solves the even system exactly
    SQ_CUDA_TRY(cudaMemsetAsync(xe, 0, fb, st));
  } else {
    sq_cg_opts eo = o;
    eo.flags = SQ_CG_DEVICE_PTRS | (guess ? SQ_CG_INITIAL_GUESS : 0u) |
               (o.flags & SQ_CG_NO_GRAPH);
    eo.stream = st;
    const double tol_e = tol * mass * std::sqrt(b2 / bt2);
    status = solve_batch_locked(ctx, gauge_id, 1, bt_c, &mass, tol_e, &eo, xe_c, &est);
    if (status < 0) return status;
    if (launch_pack(PREC_F64, g, xe_c, (size_t)3 * g.vh, xe, fb, 1, st)) return SQ_ERR_ARG;
    ctx->launches++;
  }
  // x_o = (b_o - D_oe x_e) / m
  if ((rc = ops.dslash(1, xe, t))) return rc;
  if ((rc = ops.lincomb(1.0 / mass, bo, -1.0 / mass, t, 0.0, nullptr, xo))) return rc;
  // full FP64 residual: r_o = b_o - D_oe x_e - m x_o, r_e = b_e - m x_e - D_eo x_o
  if ((rc = ops.lincomb(1.0, bo, -1.0, t, -mass, xo, ro))) return rc;
  if ((rc = ops.dslash(0, xo, t))) return rc;
  if ((rc = ops.lincomb(1.0, be, -mass, xe, -1.0, t, re))) return rc;
  if ((rc = ops.norm2(re, partial, sums + 3))) return rc;
  if ((rc = ops.norm2(ro, partial, sums + 4))) return rc;
  double *xdst = dev ? x : stage;
  if ((rc = ops.merge(xe, xo, xdst))) return rc;
  if (!dev) SQ_CUDA_TRY(cudaMemcpyAsync(x, stage, full_bytes, cudaMemcpyDeviceToHost, st));
  double rr[2];
  SQ_CUDA_TRY(cudaMemcpyAsync(rr, sums + 3, sizeof(rr), cudaMemcpyDeviceToHost, st));
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  if (stats) {
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *stats = est;
    stats->status = status;
    stats->true_residual = (b2 > 0) ? std::sqrt((rr[0] + rr[1]) / b2) : 0.0;
    stats->seconds = secs;
    stats->gflops = (secs > 0) ? 2364.0 * (double)g.vh * est.iterations / secs * 1e-9 : 0.0;
  }
  return status;
}
