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
#include <complex>
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

// out = a x + b y + c z on packed halves of precision P (z may be null)
template <int P>
__global__ void lincomb_kernel(Geom g, double a, const char *x, double b, const char *y, double c,
                               const char *z, char *out) {
  using R = typename SpinorIO<P>::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  const Vec3<R> vx = SpinorIO<P>::load(x, g.stride, i);
  const Vec3<R> vy = SpinorIO<P>::load(y, g.stride, i);
  Vec3<R> o;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    o.c[k].x = fma((R)a, vx.c[k].x, (R)b * vy.c[k].x);
    o.c[k].y = fma((R)a, vx.c[k].y, (R)b * vy.c[k].y);
  }
  if (z != nullptr) {
    const Vec3<R> vz = SpinorIO<P>::load(z, g.stride, i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o.c[k].x = fma((R)c, vz.c[k].x, o.c[k].x);
      o.c[k].y = fma((R)c, vz.c[k].y, o.c[k].y);
    }
  }
  SpinorIO<P>::store(out, g.stride, i, o);
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

// ---- whole-lattice vectors for BiCGstab: [even half][odd half], packed FP64
// halves of fb bytes each; site i < 2 vh is half i / vh, index i % vh.

template <typename R2>
__device__ __forceinline__ R2 zmul(R2 a, R2 b) {
  R2 c;
  c.x = fma(a.x, b.x, -a.y * b.y);
  c.y = fma(a.x, b.y, a.y * b.x);
  return c;
}

// out = x + a y + b z (complex a, b; z may be null) on vectors of precision
// P, arithmetic in P's real type.  With partial: also |out|^2 and
// <w, out> = sum conj(w) out (w may be null) as 3 rows of chunk partials
// (nch chunks of the 2 vh sites), accumulated in FP64.
template <int P>
__global__ void zaxpy_kernel(Geom g, size_t fb, const char *x, double2 a, const char *y,
                             double2 b, const char *z, char *out, const char *w,
                             double *partial, int nch) {
  using R = typename SpinorIO<P>::R;
  using R2 = typename C2<R>::T;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double val[3] = {0.0, 0.0, 0.0};
  if (i < 2 * g.vh) {
    const int half = i >= g.vh;
    const int j = i - half * g.vh;
    const size_t off = half * fb;
    R2 ar, br;
    ar.x = (R)a.x; ar.y = (R)a.y;
    br.x = (R)b.x; br.y = (R)b.y;
    const Vec3<R> vx = SpinorIO<P>::load(x + off, g.stride, j);
    const Vec3<R> vy = SpinorIO<P>::load(y + off, g.stride, j);
    Vec3<R> o;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const R2 t = zmul(ar, vy.c[k]);
      o.c[k].x = vx.c[k].x + t.x;
      o.c[k].y = vx.c[k].y + t.y;
    }
    if (z != nullptr) {
      const Vec3<R> vz = SpinorIO<P>::load(z + off, g.stride, j);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const R2 t = zmul(br, vz.c[k]);
        o.c[k].x += t.x;
        o.c[k].y += t.y;
      }
    }
    SpinorIO<P>::store(out + off, g.stride, j, o);
    if (partial != nullptr) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double ox = o.c[k].x, oy = o.c[k].y;
        val[0] = fma(ox, ox, fma(oy, oy, val[0]));
      }
      if (w != nullptr) {
        const Vec3<R> vw = SpinorIO<P>::load(w + off, g.stride, j);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double wx = vw.c[k].x, wy = vw.c[k].y, ox = o.c[k].x, oy = o.c[k].y;
          val[1] = fma(wx, ox, fma(wy, oy, val[1]));
          val[2] = fma(wx, oy, fma(-wy, ox, val[2]));
        }
      }
    }
  }
  if (partial != nullptr) {  // uniform
    __shared__ double smem[3 * FS_BLOCK / 32];
    chunk_reduce<3>(val, smem, partial, nch);
  }
}

// |x|^2 and <x, y> = sum conj(x) y over both parities, as 3 rows of partials.
template <int P>
__global__ void zdot_kernel(Geom g, size_t fb, const char *x, const char *y, double *partial,
                            int nch) {
  using R = typename SpinorIO<P>::R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double val[3] = {0.0, 0.0, 0.0};
  if (i < 2 * g.vh) {
    const int half = i >= g.vh;
    const int j = i - half * g.vh;
    const size_t off = half * fb;
    const Vec3<R> vx = SpinorIO<P>::load(x + off, g.stride, j);
    const Vec3<R> vy = SpinorIO<P>::load(y + off, g.stride, j);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double xx = vx.c[k].x, xy = vx.c[k].y, yx = vy.c[k].x, yy = vy.c[k].y;
      val[0] = fma(xx, xx, fma(xy, xy, val[0]));
      val[1] = fma(xx, yx, fma(xy, yy, val[1]));
      val[2] = fma(xx, yy, fma(-xy, yx, val[2]));
    }
  }
  __shared__ double smem[3 * FS_BLOCK / 32];
  chunk_reduce<3>(val, smem, partial, nch);
}

// out (precision PO) = in (precision PI) over both parities
template <int PI, int PO>
__global__ void convert_full_kernel(Geom g, const char *in, size_t fbi, char *out, size_t fbo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.vh) return;
  const int half = i >= g.vh;
  const int j = i - half * g.vh;
  using RO = typename SpinorIO<PO>::R;
  SpinorIO<PO>::store(out + half * fbo, g.stride, j,
                      convert<RO>(SpinorIO<PI>::load(in + half * fbi, g.stride, j)));
}

// x64 += xs (FP32), xs = 0, over both parities
__global__ void fold_kernel(Geom g, char *x64, size_t fb64, char *xs, size_t fb32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.vh) return;
  const int half = i >= g.vh;
  const int j = i - half * g.vh;
  Vec3<double> x = SpinorIO<PREC_F64>::load(x64 + half * fb64, g.stride, j);
  const Vec3<float> d = SpinorIO<PREC_F32>::load(xs + half * fb32, g.stride, j);
  Vec3<float> z;
  zero(z);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x.c[k].x += (double)d.c[k].x;
    x.c[k].y += (double)d.c[k].y;
  }
  SpinorIO<PREC_F64>::store(x64 + half * fb64, g.stride, j, x);
  SpinorIO<PREC_F32>::store(xs + half * fb32, g.stride, j, z);
}

// out[v] = fixed-order sum of partial row v (one block per row)
__global__ void sum_rows_kernel(const double *partial, int n, double *out) {
  __shared__ double red[32];
  const double s = block_sum_fixed(partial + (size_t)blockIdx.x * n, n, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
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
  int prec = PREC_F64;  // links and vectors of dslash, lincomb, mat, zaxpy, zdot

  int dslash(int out_parity, const char *in, char *out) {
    DslashArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = gf->g;
    a.out_parity = out_parity;
    a.links = gf->link_ptr(prec, 18, out_parity);
    a.ls = gf->scales(prec, 18);
    a.in = in;
    a.out = out;
    a.in_fb = a.out_fb = spinor_bytes(prec, gf->g.stride);
    a.nrhs = 1;
    a.gate = GATE_NONE;
    if (launch_dslash(prec, 18, 1, MODE_PLAIN, prec, a, cfg.block, st)) return SQ_ERR_ARG;
    ctx->launches++;
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
  int lincomb(double a, const char *x, double b, const char *y, double c, const char *z,
              char *out) {
    if (gf->g.vh <= 0) return SQ_OK;
    if (prec == PREC_F32)
      lincomb_kernel<PREC_F32><<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, a, x, b, y, c, z, out);
    else
      lincomb_kernel<PREC_F64><<<blocks(gf->g), FS_BLOCK, 0, st>>>(gf->g, a, x, b, y, c, z, out);
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
  // whole-lattice vectors (both halves, fb bytes apart)
  size_t fb() const { return spinor_bytes(prec, gf->g.stride); }
  int nch2() const { return (2 * gf->g.vh + CHUNK - 1) / CHUNK; }
  unsigned blocks2() const { return (unsigned)((2 * gf->g.vh + FS_BLOCK - 1) / FS_BLOCK); }
  // out = (m + D) in
  int mat(double mass, const char *in, char *out) {
    const size_t h = fb();
    int rc;
    if ((rc = dslash(0, in + h, out))) return rc;
    if ((rc = dslash(1, in, out + h))) return rc;
    if ((rc = lincomb(mass, in, 1.0, out, 0.0, nullptr, out))) return rc;
    return lincomb(mass, in + h, 1.0, out + h, 0.0, nullptr, out + h);
  }
  // out = x + a y + b z; with sums: sums[0] = |out|^2, sums[1..2] = <w, out>
  int zaxpy(const char *x, double2 a, const char *y, double2 b, const char *z, char *out,
            const char *w, double *partial, double *sums) {
    if (prec == PREC_F32)
      zaxpy_kernel<PREC_F32><<<blocks2(), FS_BLOCK, 0, st>>>(gf->g, fb(), x, a, y, b, z, out, w,
                                                             sums ? partial : nullptr, nch2());
    else
      zaxpy_kernel<PREC_F64><<<blocks2(), FS_BLOCK, 0, st>>>(gf->g, fb(), x, a, y, b, z, out, w,
                                                             sums ? partial : nullptr, nch2());
    ctx->launches++;
    if (sums) {
      sum_rows_kernel<<<3, 128, 0, st>>>(partial, nch2(), sums);
      ctx->launches++;
    }
    SQ_CUDA_TRY(cudaGetLastError());
    return SQ_OK;
  }
  // sums[0] = |x|^2, sums[1..2] = <x, y>
  int zdot(const char *x, const char *y, double *partial, double *sums) {
    if (prec == PREC_F32)
      zdot_kernel<PREC_F32><<<blocks2(), FS_BLOCK, 0, st>>>(gf->g, fb(), x, y, partial, nch2());
    else
      zdot_kernel<PREC_F64><<<blocks2(), FS_BLOCK, 0, st>>>(gf->g, fb(), x, y, partial, nch2());
    sum_rows_kernel<<<3, 128, 0, st>>>(partial, nch2(), sums);
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
  if (st == ctx->stream)  // a default stream (NULL: the legacy one): its work first
    SQ_CUDA_TRY(cudaStreamSynchronize(stream ? (cudaStream_t)stream : cudaStreamLegacy));
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
  if (st == ctx->stream)  // a default stream (NULL: the legacy one): its work first
    SQ_CUDA_TRY(cudaStreamSynchronize(o.stream ? (cudaStream_t)o.stream : cudaStreamLegacy));

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

namespace sq {
namespace {

// BiCGstab with FP32 vectors and Dslash and FP64 reliable updates (in the
// manner of Sleijpen and van der Vorst's reliable-update scheme): the
// solution increment xs accumulates in FP32 and is folded into the FP64
// solution whenever |r| falls below delta times its maximum since the last
// update, or the recursion claims convergence; r is then replaced by the
// FP64 residual b - M x, and rho by <r^, r>, and the iteration continues.
// A breakdown restarts from the FP64 residual with a new shadow residual.
int bicgstab_mixed(sq_ctx *ctx, GaugeField *gf, cudaStream_t st, const double *src, double mass,
                   double tol, const sq_cg_opts &o, bool dev, bool guess, double *x,
                   sq_cg_stats *stats, std::chrono::steady_clock::time_point t0) {
  using cplx = std::complex<double>;
  const Geom &g = gf->g;
  const size_t vol = (size_t)2 * g.vh, full_bytes = vol * 3 * 16;
  FullOps o64{ctx, gf, st, tuned_dslash(ctx, *gf, PREC_F64, 18, 1, MODE_PLAIN, st), PREC_F64};
  FullOps o32{ctx, gf, st, tuned_dslash(ctx, *gf, PREC_F32, 18, 1, MODE_PLAIN, st), PREC_F32};
  const size_t fv64 = 2 * o64.fb(), fv32 = 2 * o32.fb();
  const int nch = o64.nch2();
  FullWork w;
  w.ctx = ctx;
  w.bytes = 4 * fv64 + 7 * fv32 + (dev ? 0 : full_bytes) + ((size_t)3 * nch + 8) * sizeof(double);
  int rc = ctx->alloc(w.bytes, &w.base);
  if (rc) return rc;
  char *q = static_cast<char *>(w.base);
  char *b64 = q, *x64 = b64 + fv64, *r64 = x64 + fv64, *t64 = r64 + fv64;
  char *r = t64 + fv64, *rh = r + fv32, *p = rh + fv32, *v = p + fv32, *sv = v + fv32,
       *t = sv + fv32, *xs = t + fv32;
  char *after = xs + fv32;
  double *stage = dev ? nullptr : reinterpret_cast<double *>(after);
  double *partial = reinterpret_cast<double *>(after + (dev ? 0 : full_bytes));
  double *sums = partial + (size_t)3 * nch;
  const double2 zero = make_double2(0.0, 0.0);
  auto z2 = [](cplx c) { return make_double2(c.real(), c.imag()); };
  double h[6];
  auto fetch = [&](int n) -> int {
    SQ_CUDA_TRY(cudaMemcpyAsync(h, sums, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    SQ_CUDA_TRY(cudaStreamSynchronize(st));
    return SQ_OK;
  };
  const unsigned blocks2 = o64.blocks2();

  const double *bsrc = src;
  if (!dev) {
    SQ_CUDA_TRY(cudaMemcpyAsync(stage, src, full_bytes, cudaMemcpyHostToDevice, st));
    bsrc = stage;
  }
  if ((rc = o64.split(bsrc, b64, b64 + fv64 / 2))) return rc;
  if (guess) {
    const double *gsrc = x;
    if (!dev) {
      SQ_CUDA_TRY(cudaMemcpyAsync(stage, x, full_bytes, cudaMemcpyHostToDevice, st));
      gsrc = stage;
    }
    if ((rc = o64.split(gsrc, x64, x64 + fv64 / 2))) return rc;
  } else {
    SQ_CUDA_TRY(cudaMemsetAsync(x64, 0, fv64, st));
  }
  SQ_CUDA_TRY(cudaMemsetAsync(xs, 0, fv32, st));
  if ((rc = o64.zdot(b64, b64, partial, sums)) || (rc = fetch(1))) return rc;
  const double bn2 = h[0];
  if (!std::isfinite(bn2)) return SQ_ERR_NONFINITE;
  const double stop2 = tol * tol * bn2;
  const double delta = o.delta >= 0 ? o.delta : 0.1;

  // x64 += xs, xs = 0; r64 = b - M x64; r = r64 (FP32): returns |r64|^2 in *rr
  int nres = 0;
  auto reliable = [&](double *rr) -> int {
    ++nres;
    fold_kernel<<<blocks2, FS_BLOCK, 0, st>>>(g, x64, fv64 / 2, xs, fv32 / 2);
    ctx->launches++;
    SQ_CUDA_TRY(cudaGetLastError());
    int e;
    if ((e = o64.mat(mass, x64, t64))) return e;
    if ((e = o64.zaxpy(b64, make_double2(-1.0, 0.0), t64, zero, nullptr, r64, nullptr, partial,
                       sums)) ||
        (e = fetch(1)))
      return e;
    convert_full_kernel<PREC_F64, PREC_F32><<<blocks2, FS_BLOCK, 0, st>>>(g, r64, fv64 / 2, r,
                                                                          fv32 / 2);
    ctx->launches++;
    SQ_CUDA_TRY(cudaGetLastError());
    *rr = h[0];
    return std::isfinite(h[0]) ? SQ_OK : SQ_ERR_NONFINITE;
  };

  int it = 0, status = SQ_NOT_CONVERGED;
  double rr = 0.0;
  if (bn2 == 0) {
    SQ_CUDA_TRY(cudaMemsetAsync(x64, 0, fv64, st));
    status = SQ_OK;
  }
  for (int restart = 0; bn2 > 0 && restart < 64; ++restart) {
    if ((rc = reliable(&rr))) return rc;
    if (rr <= stop2) {
      status = SQ_OK;
      break;
    }
    if (it >= o.max_iter) break;
    // a new shadow residual
    SQ_CUDA_TRY(cudaMemcpyAsync(rh, r, fv32, cudaMemcpyDeviceToDevice, st));
    SQ_CUDA_TRY(cudaMemsetAsync(p, 0, fv32, st));
    SQ_CUDA_TRY(cudaMemsetAsync(v, 0, fv32, st));
    if ((rc = o32.zdot(rh, r, partial, sums)) || (rc = fetch(3))) return rc;
    cplx rho_old(1.0, 0.0), alpha(1.0, 0.0), omega(1.0, 0.0), rho(h[1], h[2]);
    double maxr = std::sqrt(rr);
    bool done = false;
    while (it < o.max_iter) {
      if (rho == cplx(0.0, 0.0)) break;
      const cplx beta = (rho / rho_old) * (alpha / omega);
      if ((rc = o32.zaxpy(r, z2(beta), p, z2(-beta * omega), v, p, nullptr, nullptr, nullptr)))
        return rc;
      if ((rc = o32.mat(mass, p, v))) return rc;
      if ((rc = o32.zdot(rh, v, partial, sums)) || (rc = fetch(3))) return rc;
      const cplx d(h[1], h[2]);
      if (d == cplx(0.0, 0.0)) break;
      alpha = rho / d;
      if ((rc = o32.zaxpy(r, z2(-alpha), v, zero, nullptr, sv, nullptr, partial, sums + 3)))
        return rc;
      if ((rc = o32.mat(mass, sv, t))) return rc;
      if ((rc = o32.zdot(t, sv, partial, sums)) || (rc = fetch(6))) return rc;
      ++it;
      const double ss = h[3], tt = h[0];
      const cplx ts(h[1], h[2]);
      if (!std::isfinite(ss) || !std::isfinite(tt)) return SQ_ERR_NONFINITE;
      if (ss <= stop2 || tt == 0.0) {  // x += alpha p finishes it (checked in FP64)
        if ((rc = o32.zaxpy(xs, z2(alpha), p, zero, nullptr, xs, nullptr, nullptr, nullptr)))
          return rc;
        break;
      }
      omega = ts / tt;
      if ((rc = o32.zaxpy(xs, z2(alpha), p, z2(omega), sv, xs, nullptr, nullptr, nullptr)))
        return rc;
      if ((rc = o32.zaxpy(sv, z2(-omega), t, zero, nullptr, r, rh, partial, sums)) ||
          (rc = fetch(3)))
        return rc;
      rho_old = rho;
      rho = cplx(h[1], h[2]);
      const double rn2 = h[0];
      if (omega == cplx(0.0, 0.0)) break;
      if (rn2 <= stop2 || std::sqrt(rn2) < delta * maxr) {
        if ((rc = reliable(&rr))) return rc;
        if (rr <= stop2) {
          done = true;
          status = SQ_OK;
          break;
        }
        if ((rc = o32.zdot(rh, r, partial, sums)) || (rc = fetch(3))) return rc;
        rho = cplx(h[1], h[2]);
        maxr = std::sqrt(rr);
      } else {
        maxr = std::max(maxr, std::sqrt(rn2));
      }
    }
    if (done) break;
  }
  // a final fold and FP64 residual unless the last step just made one
  if (status != SQ_OK && bn2 > 0 && (rc = reliable(&rr))) return rc;
  if (bn2 > 0 && rr <= stop2) status = SQ_OK;
  double *xdst = dev ? x : stage;
  if ((rc = o64.merge(x64, x64 + fv64 / 2, xdst))) return rc;
  if (!dev) SQ_CUDA_TRY(cudaMemcpyAsync(x, stage, full_bytes, cudaMemcpyDeviceToHost, st));
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  if (stats) {
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::memset(stats, 0, sizeof(*stats));
    stats->status = status;
    stats->iterations = it;
    stats->reliable_updates = nres;
    stats->true_residual = bn2 > 0 ? std::sqrt(rr / bn2) : 0.0;
    stats->seconds = secs;
    stats->gflops =
        (secs > 0) ? (4.0 * 1146.0 * g.vh + 100.0 * 2 * g.vh) * it / secs * 1e-9 : 0.0;
  }
  return status;
}

}  // namespace
}  // namespace sq

// BiCGstab (van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992) 631) on the
// whole-lattice matrix M = m + D itself -- the BiCG-family inverter of the
// paper's list (Sec. 3) -- in FP64.  The recurrences run on the host from
// three device reductions per iteration; the vectors stay on the device.
extern "C" int bicgstab_solve_full(sq_ctx *ctx, int gauge_id, const double *src, double mass,
                                   double tol, const sq_cg_opts *opts_in, double *x,
                                   sq_cg_stats *stats) {
  using cplx = std::complex<double>;
  if (!ctx || !src || !x) return SQ_ERR_ARG;
  if (!std::isfinite(mass) || !(tol > 0) || !std::isfinite(tol)) return SQ_ERR_ARG;
  sq_cg_opts o;
  sq_cg_opts_default(&o);
  o.precision = PREC_F64;  // without options: FP64
  if (opts_in) o = *opts_in;
  if (o.max_iter <= 0) return SQ_ERR_ARG;
  if (o.precision != PREC_F64 && o.precision != PREC_F32) return SQ_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> solve_lock(ctx->solve_mu);
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(PREC_F64, 18) || !gf->has(o.precision, 18)) return SQ_ERR_UNSUPPORTED;
  const Geom &g = gf->g;
  const bool dev = (o.flags & SQ_CG_DEVICE_PTRS) != 0;
  const bool guess = (o.flags & SQ_CG_INITIAL_GUESS) != 0;
  const size_t vol = (size_t)2 * g.vh;
  const size_t full_bytes = vol * 3 * 16;
  if (!dev && !all_finite(src, vol * 6)) return SQ_ERR_NONFINITE;
  if (!dev && guess && !all_finite(x, vol * 6)) return SQ_ERR_NONFINITE;
  cudaSetDevice(ctx->device);
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = pick_stream(ctx, o.stream);
  if (st == ctx->stream)  // a default stream (NULL: the legacy one): its work first
    SQ_CUDA_TRY(cudaStreamSynchronize(o.stream ? (cudaStream_t)o.stream : cudaStreamLegacy));

  if (o.precision == PREC_F32)
    return bicgstab_mixed(ctx, gf, st, src, mass, tol, o, dev, guess, x, stats, t0);
  FullOps ops{ctx, gf, st, tuned_dslash(ctx, *gf, PREC_F64, 18, 1, MODE_PLAIN, st)};
  const size_t fv = 2 * ops.fb();  // one whole-lattice vector
  const int nch = ops.nch2();
  FullWork w;
  w.ctx = ctx;
  w.bytes = 8 * fv + (dev ? 0 : full_bytes) + ((size_t)3 * nch + 8) * sizeof(double);
  int rc = ctx->alloc(w.bytes, &w.base);
  if (rc) return rc;
  char *base = static_cast<char *>(w.base);
  char *b = base, *xv = b + fv, *r = xv + fv, *rh = r + fv, *p = rh + fv, *v = p + fv,
       *sv = v + fv, *t = sv + fv;
  char *after = t + fv;
  double *stage = dev ? nullptr : reinterpret_cast<double *>(after);
  double *partial = reinterpret_cast<double *>(after + (dev ? 0 : full_bytes));
  double *sums = partial + (size_t)3 * nch;  // two groups of 3
  const double2 zero = make_double2(0.0, 0.0);
  auto z2 = [](cplx c) { return make_double2(c.real(), c.imag()); };
  auto fetch = [&](double *h, int n) -> int {
    SQ_CUDA_TRY(cudaMemcpyAsync(h, sums, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    SQ_CUDA_TRY(cudaStreamSynchronize(st));
    return SQ_OK;
  };

  const double *bsrc = src;
  if (!dev) {
    SQ_CUDA_TRY(cudaMemcpyAsync(stage, src, full_bytes, cudaMemcpyHostToDevice, st));
    bsrc = stage;
  }
  if ((rc = ops.split(bsrc, b, b + fv / 2))) return rc;
  if (guess) {
    const double *gsrc = x;
    if (!dev) {
      SQ_CUDA_TRY(cudaMemcpyAsync(stage, x, full_bytes, cudaMemcpyHostToDevice, st));
      gsrc = stage;
    }
    if ((rc = ops.split(gsrc, xv, xv + fv / 2))) return rc;
  } else {
    SQ_CUDA_TRY(cudaMemsetAsync(xv, 0, fv, st));
  }
  double h[6];
  if ((rc = ops.zdot(b, b, partial, sums)) || (rc = fetch(h, 1))) return rc;
  const double bn2 = h[0];
  if (!std::isfinite(bn2)) return SQ_ERR_NONFINITE;
  const double stop2 = tol * tol * bn2;

  int it = 0, status = SQ_NOT_CONVERGED, nres = 0;
  double res = 0.0;
  if (bn2 == 0) {  // M x = 0: x = 0
    SQ_CUDA_TRY(cudaMemsetAsync(xv, 0, fv, st));
    status = SQ_OK;
  }
  // r = b - M x; a restart begins here whenever the recursion stops
  for (int restart = 0; bn2 > 0 && restart < 64; ++restart) {
    ++nres;
    if ((rc = ops.mat(mass, xv, t))) return rc;
    if ((rc = ops.zaxpy(b, make_double2(-1.0, 0.0), t, zero, nullptr, r, nullptr, partial, sums)) ||
        (rc = fetch(h, 1)))
      return rc;
    res = std::sqrt(h[0] / bn2);
    if (!std::isfinite(res)) return SQ_ERR_NONFINITE;
    if (h[0] <= stop2) {
      status = SQ_OK;
      break;
    }
    if (it >= o.max_iter) break;
    SQ_CUDA_TRY(cudaMemcpyAsync(rh, r, fv, cudaMemcpyDeviceToDevice, st));
    SQ_CUDA_TRY(cudaMemsetAsync(p, 0, fv, st));
    SQ_CUDA_TRY(cudaMemsetAsync(v, 0, fv, st));
    cplx rho_old(1.0, 0.0), alpha(1.0, 0.0), omega(1.0, 0.0), rho(h[0], 0.0);
    while (it < o.max_iter) {
      if (rho == cplx(0.0, 0.0)) break;
      const cplx beta = (rho / rho_old) * (alpha / omega);
      // p = r + beta (p - omega v)
      if ((rc = ops.zaxpy(r, z2(beta), p, z2(-beta * omega), v, p, nullptr, nullptr, nullptr)))
        return rc;
      if ((rc = ops.mat(mass, p, v))) return rc;
      if ((rc = ops.zdot(rh, v, partial, sums)) || (rc = fetch(h, 3))) return rc;
      const cplx d(h[1], h[2]);
      if (d == cplx(0.0, 0.0)) break;
      alpha = rho / d;
      // s = r - alpha v, |s|^2
      if ((rc = ops.zaxpy(r, z2(-alpha), v, zero, nullptr, sv, nullptr, partial, sums + 3)))
        return rc;
      if ((rc = ops.mat(mass, sv, t))) return rc;
      if ((rc = ops.zdot(t, sv, partial, sums)) || (rc = fetch(h, 6))) return rc;
      ++it;
      const double ss = h[3], tt = h[0];
      const cplx ts(h[1], h[2]);
      if (!std::isfinite(ss) || !std::isfinite(tt)) return SQ_ERR_NONFINITE;
      if (ss <= stop2 || tt == 0.0) {  // x += alpha p finishes it
        if ((rc = ops.zaxpy(xv, z2(alpha), p, zero, nullptr, xv, nullptr, nullptr, nullptr)))
          return rc;
        break;
      }
      omega = ts / tt;
      // x += alpha p + omega s;  r = s - omega t, |r|^2, <r^, r>
      if ((rc = ops.zaxpy(xv, z2(alpha), p, z2(omega), sv, xv, nullptr, nullptr, nullptr)))
        return rc;
      if ((rc = ops.zaxpy(sv, z2(-omega), t, zero, nullptr, r, rh, partial, sums)) ||
          (rc = fetch(h, 3)))
        return rc;
      rho_old = rho;
      rho = cplx(h[1], h[2]);
      if (h[0] <= stop2 || omega == cplx(0.0, 0.0)) break;
    }
  }
  double *xdst = dev ? x : stage;
  if ((rc = ops.merge(xv, xv + fv / 2, xdst))) return rc;
  if (!dev) SQ_CUDA_TRY(cudaMemcpyAsync(x, stage, full_bytes, cudaMemcpyDeviceToHost, st));
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  if (stats) {
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::memset(stats, 0, sizeof(*stats));
    stats->status = status;
    stats->iterations = it;
    stats->reliable_updates = nres;  // FP64 residuals b - M x recomputed
    stats->true_residual = res;
    stats->seconds = secs;
    // two M = m + D products (4 Dslash) and ~ 100 flops of BLAS per site
    stats->gflops =
        (secs > 0) ? (4.0 * 1146.0 * g.vh + 100.0 * 2 * g.vh) * it / secs * 1e-9 : 0.0;
  }
  return status;
}
