// Fat and long links from thin links on the GPU, in FP64.
//
// The paper's lattices are MILC asqtad ensembles (Sec. 2, Fig. 1), whose fat
// and Naik links come from the thin gauge links by path sums.  This file
// builds the benchmark workloads' recipe of them from thin links U:
//   F_mu(x) = c1 [ U_mu(x) + w sum_{nu != mu} ( U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
//                + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ) ] / (1 + 6w),
//   L_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu),
// one thread per (site, direction), periodic neighbours, links in the
// canonical host layout [site_lex][mu][row][col] complex128.  The work is
// FP64 arithmetic (about 2800 flops per link against 432 bytes of traffic),
// so it is bound by the FP64 units, not by HBM.
#include <cmath>
#include <cstring>

#include "sq_host.h"

namespace sq {
namespace {

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// c = op(a) op(b), op = identity or dagger; each complex term is four FMAs
// into the accumulator (the FP64 units bound these kernels).
template <bool DA, bool DB>
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 t = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = DA ? cconj(a.e[3 * k + i]) : a.e[3 * i + k];
        const double2 y = DB ? cconj(b.e[3 * j + k]) : b.e[3 * k + j];
        t.x = fma(x.x, y.x, t.x);
        t.x = fma(-x.y, y.y, t.x);
        t.y = fma(x.x, y.y, t.y);
        t.y = fma(x.y, y.x, t.y);
      }
      c.e[3 * i + j] = t;
    }
  }
  return c;
}

struct FatGeom {
  int L[4];
  long st[4];
  long vol;
};

__device__ __forceinline__ M3 load_link(const double2 *u, long s, int mu) {
  M3 m;
  const double2 *p = u + (s * 4 + mu) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.e[e] = __ldg(p + e);
  return m;
}

// site of x + d * mu_hat, periodic (|d| <= 2)
__device__ __forceinline__ long shift(const FatGeom &g, long s, const int c[4], int mu, int d) {
  int v = c[mu] + d;
  while (v < 0) v += g.L[mu];
  while (v >= g.L[mu]) v -= g.L[mu];
  return s + (long)(v - c[mu]) * g.st[mu];
}

__global__ void __launch_bounds__(128) fatten_kernel(FatGeom g, const double2 *u, double c1,
                                                     double c3, double w, double2 *fat,
                                                     double2 *lng) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.vol) return;
  const long s = idx >> 2;
  const int mu = (int)(idx & 3);
  int c[4];
  {
    long r = s;
    c[0] = (int)(r % g.L[0]); r /= g.L[0];
    c[1] = (int)(r % g.L[1]); r /= g.L[1];
    c[2] = (int)(r % g.L[2]);
    c[3] = (int)(r / g.L[2]);
  }
  const long xpm = shift(g, s, c, mu, 1);
  const M3 umu = load_link(u, s, mu);
  M3 st;
#pragma unroll
  for (int e = 0; e < 9; ++e) st.e[e] = make_double2(0.0, 0.0);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    // up staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
    const long xpn = shift(g, s, c, nu, 1);
    M3 t = mul<false, false>(load_link(u, s, nu), load_link(u, xpn, mu));
    M3 up = mul<false, true>(t, load_link(u, xpm, nu));
    // down staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
    const long xmn = shift(g, s, c, nu, -1);
    int cm[4] = {c[0], c[1], c[2], c[3]};
    cm[nu] = (c[nu] == 0) ? g.L[nu] - 1 : c[nu] - 1;
    const long xmnpm = shift(g, xmn, cm, mu, 1);
    t = mul<true, false>(load_link(u, xmn, nu), load_link(u, xmn, mu));
    M3 dn = mul<false, false>(t, load_link(u, xmnpm, nu));
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      st.e[e].x += up.e[e].x + dn.e[e].x;
      st.e[e].y += up.e[e].y + dn.e[e].y;
    }
  }
  const double k = c1 / (1.0 + 6.0 * w);
  double2 *f = fat + idx * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e)
    f[e] = make_double2(k * fma(w, st.e[e].x, umu.e[e].x), k * fma(w, st.e[e].y, umu.e[e].y));
  const long xp2m = shift(g, s, c, mu, 2);
  const M3 n = mul<false, false>(mul<false, false>(umu, load_link(u, xpm, mu)),
                                 load_link(u, xp2m, mu));
  double2 *l = lng + idx * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) l[e] = make_double2(c3 * n.e[e].x, c3 * n.e[e].y);
}

// ---------------------------------------------------------------- asqtad
// The asqtad action's fat link (MILC's path set): the one-link term, the 6
// three-link staples, 24 five-link and 48 seven-link staples and 6 Lepage
// terms, each a product of links along its path, weighted by its
// coefficient; the Naik link is c_N U U U.  Paths, for direction mu, with
// nu, rho, sigma distinct and != mu and every sign s, r, q = +-1:
//   3-staple  (s nu) mu (-s nu)
//   5-staple  (r rho)(s nu) mu (-s nu)(-r rho)
//   7-staple  (q sg)(r rho)(s nu) mu (-s nu)(-r rho)(-q sg)
//   Lepage    (s nu)(s nu) mu (-s nu)(-s nu)
// A hop +d at y multiplies by U_d(y), a hop -d by U_d(y - d)^dag.
//
// Every longer path is a staple around a shorter one, so the paths are built
// as whole-lattice fields, each level from the one before:
//   S3 = St_{s nu}[U_mu],  Lepage = St_{s nu}[S3],  S5 = St_{r rho}[S3],
//   S7 = St_{q sg}[S5],
//   St_{s nu}[W](x) = h(x) W(x + s nu) h(x + mu)^dag,
//   h(y) = U_nu(y) (s = +1) or U_nu(y - nu)^dag (s = -1),
// two SU(3) products per staple: 168 per link for the fat link instead of
// 422 for every path multiplied out on its own.  One kernel per staple
// field, one thread per site; S3 and S5 live in device scratch.

struct StapleArgs {
  FatGeom g;
  const double2 *u;   // thin links [site][4][9]
  const double2 *w;   // the extended link W(y) at w + y * w_stride
  long w_stride;      // 36 (a direction of the links) or 9 (a field)
  int mu, nu, s;
  int both;           // add St of s and of -s (the two closings of one S5)
  double c;
  double2 *acc;       // acc(x) at acc + x * 36 (the fat link of direction mu)
  double2 *out;       // St(x) at out + x * 9, or null
};

__global__ void __launch_bounds__(128) staple_kernel(StapleArgs a) {
  const long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.g.vol) return;
  int c[4];
  {
    long r = x;
    c[0] = (int)(r % a.g.L[0]); r /= a.g.L[0];
    c[1] = (int)(r % a.g.L[1]); r /= a.g.L[1];
    c[2] = (int)(r % a.g.L[2]);
    c[3] = (int)(r / a.g.L[2]);
  }
  const long xpm = shift(a.g, x, c, a.mu, 1);
  int cm[4] = {c[0], c[1], c[2], c[3]};
  cm[a.mu] = (c[a.mu] + 1 == a.g.L[a.mu]) ? 0 : c[a.mu] + 1;
  M3 sum;
#pragma unroll
  for (int e = 0; e < 9; ++e) sum.e[e] = make_double2(0.0, 0.0);
  for (int k = 0; k < (a.both ? 2 : 1); ++k) {
    const int s = k ? -a.s : a.s;
    const long xs = shift(a.g, x, c, a.nu, s);     // x + s nu
    M3 w;
#pragma unroll
    for (int e = 0; e < 9; ++e) w.e[e] = __ldg(a.w + xs * a.w_stride + e);
    M3 t;
    if (s > 0) {  // U_nu(x) W(x + nu) U_nu(x + mu)^dag
      t = mul<false, true>(mul<false, false>(load_link(a.u, x, a.nu), w),
                           load_link(a.u, xpm, a.nu));
    } else {      // U_nu(x - nu)^dag W(x - nu) U_nu(x - nu + mu)
      const long xmnpm = shift(a.g, xpm, cm, a.nu, -1);
      t = mul<false, false>(mul<true, false>(load_link(a.u, xs, a.nu), w),
                            load_link(a.u, xmnpm, a.nu));
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      sum.e[e].x += t.e[e].x;
      sum.e[e].y += t.e[e].y;
    }
  }
  if (a.out != nullptr) {
    double2 *o = a.out + x * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) o[e] = sum.e[e];
  }
  double2 *f = a.acc + x * 36;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double2 v = f[e];
    f[e] = make_double2(fma(a.c, sum.e[e].x, v.x), fma(a.c, sum.e[e].y, v.y));
  }
}

// fat = c_one U (every direction); lng = c_N U_mu(x) U_mu(x+mu) U_mu(x+2mu)
__global__ void __launch_bounds__(128) one_link_naik_kernel(FatGeom g, const double2 *u,
                                                            double c_one, double c_naik,
                                                            double2 *fat, double2 *lng) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * g.vol) return;
  const long x = idx >> 2;
  const int mu = (int)(idx & 3);
  int c[4];
  {
    long r = x;
    c[0] = (int)(r % g.L[0]); r /= g.L[0];
    c[1] = (int)(r % g.L[1]); r /= g.L[1];
    c[2] = (int)(r % g.L[2]);
    c[3] = (int)(r / g.L[2]);
  }
  const M3 l = load_link(u, x, mu);
  double2 *f = fat + idx * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) f[e] = make_double2(c_one * l.e[e].x, c_one * l.e[e].y);
  const M3 n = mul<false, false>(mul<false, false>(l, load_link(u, shift(g, x, c, mu, 1), mu)),
                                 load_link(u, shift(g, x, c, mu, 2), mu));
  double2 *o = lng + idx * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) o[e] = make_double2(c_naik * n.e[e].x, c_naik * n.e[e].y);
}

struct AsqtadCoeffs {
  double one, three, five, seven, lepage, naik;
};

int launch_fatten(const int dims[4], long vol, const double *thin, double c1, double c3, double w,
                  double *fat, double *lng, cudaStream_t st) {
  FatGeom g;
  for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
  g.st[0] = 1;
  g.st[1] = dims[0];
  g.st[2] = (long)dims[0] * dims[1];
  g.st[3] = (long)dims[0] * dims[1] * dims[2];
  g.vol = vol;
  const long n = 4 * vol;
  fatten_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
      g, reinterpret_cast<const double2 *>(thin), c1, c3, w, reinterpret_cast<double2 *>(fat),
      reinterpret_cast<double2 *>(lng));
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}

FatGeom make_fat_geom(const int dims[4], long vol) {
  FatGeom g;
  for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
  g.st[0] = 1;
  g.st[1] = dims[0];
  g.st[2] = (long)dims[0] * dims[1];
  g.st[3] = (long)dims[0] * dims[1] * dims[2];
  g.vol = vol;
  return g;
}

}  // namespace

int check_lattice_dims(const int dims[4], long *vol) {
  long v = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || (dims[mu] & 1)) return SQ_ERR_ARG;
    v *= dims[mu];
    if (v > (1L << 30)) return SQ_ERR_ARG;
  }
  *vol = v;
  return SQ_OK;
}

}  // namespace sq

using namespace sq;

extern "C" int gauge_fatten_asqtad(sq_ctx *ctx, const int dims[4], const double *thin_dev,
                                   const double coeffs[6], double *fat_dev, double *lng_dev,
                                   void *stream) {
  if (!ctx || !dims || !thin_dev || !coeffs || !fat_dev || !lng_dev) return SQ_ERR_ARG;
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(coeffs[k])) return SQ_ERR_ARG;
  long vol;
  int rc = check_lattice_dims(dims, &vol);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamLegacy;  // NULL: default stream
  const AsqtadCoeffs k{coeffs[0], coeffs[1], coeffs[2], coeffs[3], coeffs[4], coeffs[5]};
  const FatGeom g = make_fat_geom(dims, vol);
  const double2 *u = reinterpret_cast<const double2 *>(thin_dev);
  double2 *fat = reinterpret_cast<double2 *>(fat_dev);
  one_link_naik_kernel<<<(unsigned)((4 * vol + 127) / 128), 128, 0, st>>>(
      g, u, k.one, k.naik, fat, reinterpret_cast<double2 *>(lng_dev));
  SQ_CUDA_TRY(cudaGetLastError());
  uint64_t launches = 1;
  void *scratch = nullptr;  // S3 and S5 fields, stream-ordered
  SQ_CUDA_TRY(cudaMallocAsync(&scratch, sizeof(double2) * 18 * (size_t)vol, st));
  double2 *s3 = static_cast<double2 *>(scratch), *s5 = s3 + 9 * vol;
  const unsigned blocks = (unsigned)((vol + 127) / 128);
  cudaError_t e = cudaSuccess;
  auto staple = [&](const double2 *w, long w_stride, int mu, int nu, int s, int both, double c,
                    double2 *out) {
    if (e != cudaSuccess) return;
    StapleArgs a{g, u, w, w_stride, mu, nu, s, both, c, fat + mu * 9, out};
    staple_kernel<<<blocks, 128, 0, st>>>(a);
    e = cudaGetLastError();
    ++launches;
  };
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      for (int s = -1; s <= 1; s += 2) {
        staple(u + mu * 9, 36, mu, nu, s, 0, k.three, s3);   // 3-staple
        staple(s3, 9, mu, nu, s, 0, k.lepage, nullptr);     // Lepage
        for (int rho = 0; rho < 4; ++rho) {
          if (rho == mu || rho == nu) continue;
          for (int r = -1; r <= 1; r += 2) {
            staple(s3, 9, mu, rho, r, 0, k.five, s5);       // 5-staple
            const int sg = 6 - mu - nu - rho;
            staple(s5, 9, mu, sg, -1, 1, k.seven, nullptr);  // both 7-staples
          }
        }
      }
    }
  cudaFreeAsync(scratch, st);
  ctx->launches += launches;
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "asqtad staple kernels", __FILE__, __LINE__);
    return SQ_ERR_CUDA;
  }
  return SQ_OK;
}

extern "C" int gauge_fatten(sq_ctx *ctx, const int dims[4], const double *thin_dev, double c1,
                            double c3, double staple_weight, double *fat_dev, double *lng_dev,
                            void *stream) {
  if (!ctx || !dims || !thin_dev || !fat_dev || !lng_dev) return SQ_ERR_ARG;
  if (!std::isfinite(c1) || !std::isfinite(c3) || !std::isfinite(staple_weight) ||
      1.0 + 6.0 * staple_weight == 0.0)
    return SQ_ERR_ARG;
  long vol;
  int rc = check_lattice_dims(dims, &vol);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamLegacy;  // NULL: default stream
  rc = launch_fatten(dims, vol, thin_dev, c1, c3, staple_weight, fat_dev, lng_dev, st);
  if (rc == SQ_OK) ctx->launches++;
  return rc;
}

extern "C" int gauge_load_thin(sq_ctx *ctx, const int dims[4], const double *thin, double c1,
                               double c3, double staple_weight, unsigned flags, int *gauge_id) {
  if (!ctx || !dims || !thin || !gauge_id) return SQ_ERR_ARG;
  long vol;
  int rc = check_lattice_dims(dims, &vol);
  if (rc) return rc;
  const size_t nbytes = (size_t)vol * 4 * 9 * 16;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  // staging of thin, fat and long links, freed before return: outside the budget
  void *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 3 * nbytes);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "cudaMalloc(link staging)", __FILE__, __LINE__);
    return SQ_ERR_OOM;
  }
  double *du = static_cast<double *>(buf);
  double *df = du + (size_t)vol * 72, *dl = df + (size_t)vol * 72;
  const double *src = thin;
  if (!(flags & SQ_GAUGE_DEVICE_PTRS)) {
    for (size_t k = 0; k < (size_t)vol * 72; ++k)
      if (!std::isfinite(thin[k])) {
        cudaFree(buf);
        return SQ_ERR_NONFINITE;
      }
    e = cudaMemcpyAsync(du, thin, nbytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFree(buf);
      set_last_cuda_error(e, "cudaMemcpyAsync(thin links)", __FILE__, __LINE__);
      return SQ_ERR_CUDA;
    }
    src = du;
  }
  rc = gauge_fatten(ctx, dims, src, c1, c3, staple_weight, df, dl, st);
  if (rc == SQ_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "gauge_fatten", __FILE__, __LINE__);
      rc = SQ_ERR_CUDA;
    }
  }
  if (rc == SQ_OK) rc = gauge_load(ctx, dims, df, dl, flags | SQ_GAUGE_DEVICE_PTRS, gauge_id);
  cudaFree(buf);
  return rc;
}
