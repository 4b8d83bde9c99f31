// gauge_load's device work: statistics of the input links (16-bit scales,
// 12-real reconstruction residual) and the pack into the Dslash's per-site
// hop-matrix planes for every precision and link format.
#include "sq_device.cuh"
#include "gauge_pack.h"

namespace sq {

namespace {

using cd = double2;

__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ cd cmul(cd a, cd b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One link matrix (9 complex) at [site_lex][mu]
__device__ __forceinline__ void load_link(const cd *u, long s, int mu, cd m[9]) {
  const cd *p = u + (s * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = p[k];
}

__device__ __forceinline__ void dagger(cd m[9]) {
  cd t[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) t[3 * r + c] = make_double2(m[3 * c + r].x, -m[3 * c + r].y);
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = t[k];
}

__global__ void gauge_stats_kernel(const cd *fat, const cd *lng, long nlinks, double inv_s,
                                   unsigned long long *out /* [fat max, long max, recon err] */) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double fm = 0, lm = 0, err = 0;
  for (; k < nlinks; k += (long)gridDim.x * blockDim.x) {
    const cd *f = fat + k * 9;
    const cd *l = lng + k * 9;
    cd w[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      fm = fmax(fm, fmax(fabs(f[e].x), fabs(f[e].y)));
      w[e] = l[e];
      lm = fmax(lm, fmax(fabs(w[e].x), fabs(w[e].y)));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      cd x = cmul(w[c1], w[3 + c2]);
      cd y = cmul(w[c2], w[3 + c1]);
      cd r = make_double2((x.x - y.x) * inv_s, -(x.y - y.y) * inv_s);
      err = fmax(err, fmax(fabs(r.x - w[6 + c].x), fabs(r.y - w[6 + c].y)));
    }
  }
  atomic_max_pos(out + 0, fm);
  atomic_max_pos(out + 1, lm);
  atomic_max_pos(out + 2, err);
}

__device__ __forceinline__ uint32_t link_word(cd v, float inv) {
  return encode_word(__double2float_rn(v.x), __double2float_rn(v.y), inv);
}

// Writes the fat pair (F_mu(x), F_mu(x-mu)^dag) and the long pair
// (L_mu(x), L_mu(x-3mu)^dag) of one site in layout <PREC, RECON>.
template <int PREC, int RECON>
__device__ void store_pairs(char *links, int S, int i, int mu, const cd ff[9], const cd fb[9],
                            const cd lf[9], const cd lb[9], const PackScales &ps) {
  using LL = LinkLayout<PREC, RECON>;
  char *fat = links + (size_t)mu * LL::mu_bytes * S;
  char *lng = fat + (size_t)LL::fat_bytes * S;
  const int nl = (RECON == 18) ? 9 : 6;  // stored elements per long link
  if constexpr (PREC == PREC_F64) {
    double2 *pf = reinterpret_cast<double2 *>(fat);
    double2 *pl = reinterpret_cast<double2 *>(lng);
    for (int k = 0; k < 9; ++k) {
      pf[(size_t)k * S + i] = ff[k];
      pf[(size_t)(9 + k) * S + i] = fb[k];
    }
    for (int k = 0; k < nl; ++k) {
      pl[(size_t)k * S + i] = lf[k];
      pl[(size_t)(nl + k) * S + i] = lb[k];
    }
  } else if constexpr (PREC == PREC_F32) {
    float f[36];
    for (int k = 0; k < 9; ++k) {
      f[2 * k] = __double2float_rn(ff[k].x); f[2 * k + 1] = __double2float_rn(ff[k].y);
      f[18 + 2 * k] = __double2float_rn(fb[k].x); f[19 + 2 * k] = __double2float_rn(fb[k].y);
    }
    float4 *pf = reinterpret_cast<float4 *>(fat);
    for (int k = 0; k < 9; ++k)
      pf[(size_t)k * S + i] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    for (int k = 0; k < nl; ++k) {
      f[2 * k] = __double2float_rn(lf[k].x); f[2 * k + 1] = __double2float_rn(lf[k].y);
      f[2 * nl + 2 * k] = __double2float_rn(lb[k].x);
      f[2 * nl + 2 * k + 1] = __double2float_rn(lb[k].y);
    }
    float4 *pl = reinterpret_cast<float4 *>(lng);
    for (int k = 0; k < nl; ++k)
      pl[(size_t)k * S + i] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
  } else {
    uint32_t w[18];
    for (int k = 0; k < 9; ++k) {
      w[k] = link_word(ff[k], ps.fat_inv);
      w[9 + k] = link_word(fb[k], ps.fat_inv);
    }
    uint4 *pf = reinterpret_cast<uint4 *>(fat);
    for (int k = 0; k < 4; ++k)
      pf[(size_t)k * S + i] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    reinterpret_cast<uint2 *>(fat + (size_t)64 * S)[i] = make_uint2(w[16], w[17]);
    for (int k = 0; k < nl; ++k) {
      w[k] = link_word(lf[k], ps.long_inv);
      w[nl + k] = link_word(lb[k], ps.long_inv);
    }
    uint4 *pl = reinterpret_cast<uint4 *>(lng);
    if (RECON == 18) {
      for (int k = 0; k < 4; ++k)
        pl[(size_t)k * S + i] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
      reinterpret_cast<uint2 *>(lng + (size_t)64 * S)[i] = make_uint2(w[16], w[17]);
    } else {
      for (int k = 0; k < 3; ++k)
        pl[(size_t)k * S + i] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    }
  }
}

template <int PREC, int RECON>
__global__ void gauge_pack_kernel(Geom g, const cd *fat, const cd *lng, char *links_even,
                                  char *links_odd, PackScales ps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int parity = blockIdx.y;
  if (i >= g.vh) return;
  char *links = parity ? links_odd : links_even;
  SiteCoords sc = site_coords(g, parity, i);
  for (int mu = 0; mu < 4; ++mu) {
    int c = sc.c[mu];
    int L = g.L[mu];
    long x = sc.lex;
    long xm1 = x + (long)(((c - 1 + L) % L) - c) * g.st[mu];
    long xm3 = x + (long)(((c - 3 + 3 * L) % L) - c) * g.st[mu];
    cd ff[9], fb[9], lf[9], lb[9];
    load_link(fat, x, mu, ff);
    load_link(fat, xm1, mu, fb);
    dagger(fb);
    load_link(lng, x, mu, lf);
    load_link(lng, xm3, mu, lb);
    dagger(lb);
    store_pairs<PREC, RECON>(links, g.stride, i, mu, ff, fb, lf, lb, ps);
  }
}

}  // namespace

int launch_gauge_stats(const double *fat, const double *lng, long nlinks, double inv_s,
                       unsigned long long *out, cudaStream_t st) {
  gauge_stats_kernel<<<1216, 256, 0, st>>>(reinterpret_cast<const cd *>(fat),
                                           reinterpret_cast<const cd *>(lng), nlinks, inv_s, out);
  return 0;
}

int launch_gauge_pack(int prec, int recon, const Geom &g, const double *fat, const double *lng,
                      void *links_even, void *links_odd, const PackScales &ps, cudaStream_t st) {
  if (g.vh <= 0) return 0;
  dim3 grid((g.vh + 127) / 128, 2);
  const cd *f = reinterpret_cast<const cd *>(fat);
  const cd *l = reinterpret_cast<const cd *>(lng);
  char *e = static_cast<char *>(links_even), *o = static_cast<char *>(links_odd);
#define SQ_GP(P, RC) gauge_pack_kernel<P, RC><<<grid, 128, 0, st>>>(g, f, l, e, o, ps)
  if (prec == PREC_F64 && recon == 18) SQ_GP(PREC_F64, 18);
  else if (prec == PREC_F64 && recon == 12) SQ_GP(PREC_F64, 12);
  else if (prec == PREC_F32 && recon == 18) SQ_GP(PREC_F32, 18);
  else if (prec == PREC_F32 && recon == 12) SQ_GP(PREC_F32, 12);
  else if (prec == PREC_I16 && recon == 18) SQ_GP(PREC_I16, 18);
  else if (prec == PREC_I16 && recon == 12) SQ_GP(PREC_I16, 12);
  else return -1;
#undef SQ_GP
  return 0;
}

size_t link_site_bytes(int prec, int recon) {
#define SQ_LB(P, RC) if (prec == P && recon == RC) return LinkLayout<P, RC>::site_bytes;
  SQ_LB(PREC_F64, 18) SQ_LB(PREC_F64, 12) SQ_LB(PREC_F32, 18) SQ_LB(PREC_F32, 12)
  SQ_LB(PREC_I16, 18) SQ_LB(PREC_I16, 12)
#undef SQ_LB
  return 0;
}

}  // namespace sq
