// Device-side building blocks of the asqtad CG: lattice geometry, the packed
// field layouts, link/colour-vector loads and stores per precision, SU(3)
// mat-vecs and the fixed-order (deterministic) reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sq_types.h"

namespace sq {

// ----------------------------------------------------------------- geometry
//
// Sites of one parity are ranked by i = site_lex / 2 (Lx even), so for a
// parity p: x = 2*(i % (Lx/2)) + ((p + y + z + t) & 1).

struct SiteCoords {
  int c[4];
  int lex;
};

__device__ __forceinline__ uint32_t geom_div(const Geom &g, int k, uint32_t n) {
  uint32_t t = __umulhi(n, g.div_m[k]);
  return (t + ((n - t) >> g.div_s1[k])) >> g.div_s2[k];
}

__device__ __forceinline__ SiteCoords site_coords(const Geom &g, int parity, int i) {
  SiteCoords s;
  uint32_t r = geom_div(g, 0, (uint32_t)i);
  const int xh = i - (int)r * g.lxh;
  uint32_t r2 = geom_div(g, 1, r);
  s.c[1] = (int)(r - r2 * (uint32_t)g.L[1]);
  uint32_t r3 = geom_div(g, 2, r2);
  s.c[2] = (int)(r2 - r3 * (uint32_t)g.L[2]);
  s.c[3] = (int)r3;
  s.c[0] = 2 * xh + ((parity + s.c[1] + s.c[2] + s.c[3]) & 1);
  s.lex = s.c[0] + g.L[0] * (s.c[1] + g.L[1] * (s.c[2] + g.L[2] * s.c[3]));
  return s;
}

// Half-lattice index of x + d*mu_hat (periodic) and the boundary sign
// (-1 for each wrap around t when time is antiperiodic).
__device__ __forceinline__ int hop_index(const Geom &g, const SiteCoords &s, int mu, int d,
                                         float &sign) {
  int L = g.L[mu];
  int c = s.c[mu] + d;
  int wraps = 0;
  while (c < 0) { c += L; ++wraps; }
  while (c >= L) { c -= L; ++wraps; }
  sign = (mu == 3 && g.t_antiperiodic && (wraps & 1)) ? -1.f : 1.f;
  return (s.lex + (c - s.c[mu]) * g.st[mu]) >> 1;
}

// Same as hop_index for a hop length D known at compile time (|D| <= 3,
// L >= 2: at most two wraps, only in the direction of the hop).
template <int D>
__device__ __forceinline__ int hop(const Geom &g, const SiteCoords &s, int mu, float &sign) {
  const int L = g.L[mu];
  int c = s.c[mu] + D;
  bool w1, w2 = false;
  if constexpr (D > 0) {
    w1 = c >= L;
    c -= w1 ? L : 0;
    if constexpr (D > 1) { w2 = c >= L; c -= w2 ? L : 0; }
  } else {
    w1 = c < 0;
    c += w1 ? L : 0;
    if constexpr (D < -1) { w2 = c < 0; c += w2 ? L : 0; }
  }
  sign = (mu == 3 && g.t_antiperiodic && (w1 != w2)) ? -1.f : 1.f;
  return (s.lex + (c - s.c[mu]) * g.st[mu]) >> 1;
}

// eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})
__device__ __forceinline__ float eta_sign(const SiteCoords &s, int mu) {
  int sum = 0;
#pragma unroll
  for (int nu = 0; nu < 3; ++nu) sum += (nu < mu) ? s.c[nu] : 0;
  return (sum & 1) ? -1.f : 1.f;
}

// ------------------------------------------------- dependent launches
// The CG's kernels are launched with programmatic stream serialization: the
// next kernel may be launched while the previous one drains, and waits in
// griddep_wait() until that kernel has completed and its writes are visible.
// Nothing written by the previous kernel may be touched before that call.
// griddep_launch_dependents() allows the next kernel to launch once every
// block of this one has passed it.  Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ----------------------------------------------------------- complex types

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R> struct Vec3 { typename C2<R>::T c[3]; };
template <typename R> struct Mat3 { typename C2<R>::T e[9]; };  // row-major

template <typename R>
__device__ __forceinline__ void zero(Vec3<R> &v) {
#pragma unroll
  for (int k = 0; k < 3; ++k) { v.c[k].x = 0; v.c[k].y = 0; }
}

// acc += s * (M v), s = +-1 folded into the FMAs by the caller's choice of sign
template <typename R>
__device__ __forceinline__ void mat_vec_acc(Vec3<R> &acc, const Mat3<R> &m, const Vec3<R> &v) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc.c[r].x = fma(m.e[3 * r + c].x, v.c[c].x, acc.c[r].x);
      acc.c[r].x = fma(-m.e[3 * r + c].y, v.c[c].y, acc.c[r].x);
      acc.c[r].y = fma(m.e[3 * r + c].x, v.c[c].y, acc.c[r].y);
      acc.c[r].y = fma(m.e[3 * r + c].y, v.c[c].x, acc.c[r].y);
    }
  }
}

// row2 = f * conj(row0 x row1): rebuilds the third row of f-scaled SU(3)
template <typename R>
__device__ __forceinline__ void reconstruct_row2(Mat3<R> &m, R f) {
  using T = typename C2<R>::T;
  const T *a = &m.e[0], *b = &m.e[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    // (a x b)_k = a_k1 b_k2 - a_k2 b_k1
    R re = a[k1].x * b[k2].x - a[k1].y * b[k2].y - (a[k2].x * b[k1].x - a[k2].y * b[k1].y);
    R im = a[k1].x * b[k2].y + a[k1].y * b[k2].x - (a[k2].x * b[k1].y + a[k2].y * b[k1].x);
    m.e[6 + k].x = f * re;
    m.e[6 + k].y = -f * im;
  }
}

// ------------------------------------------------------- read-only loads
// Links stream from HBM once per Dslash: keep them out of L1, and mark them
// evict-first in L2 so that the stream does not push out the colour vectors
// every kernel of a CG iteration reads again (a few MB per field, resident
// in L2).  Colour vectors are gathered 16 times per site: let them allocate
// in L1.

// keep = true: another tile of the same launch reads these links again soon
// (its blocks are adjacent in the launch order), so they stay evict-normal;
// the last reader marks them evict-first.
__device__ __forceinline__ uint64_t l2_link_policy(bool keep) {
  uint64_t p;
  if (keep) asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  else asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ float4 ld_stream_f4(const void *p, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_stream_d2(const void *p, uint64_t pol) {
  double2 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
      : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const void *p, uint64_t pol) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ld_stream_u2(const void *p, uint64_t pol) {
  uint2 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
      : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
  return v;
}

// ------------------------------------------------------------- int16 codes
// A 16-bit code is stored excess-32768; a 32-bit word holds (re, im) codes.
// Decoding: splice the code under the exponent of 2^23 and subtract
// 2^23 + 32768 (exact), avoiding the integer-to-float conversion unit.

__device__ __forceinline__ float2 decode_word(uint32_t w) {
  float re = __int_as_float(__byte_perm(w, 0x4B00u, 0x5410u)) - 8421376.f;
  float im = __int_as_float(__byte_perm(w, 0x4B00u, 0x5432u)) - 8421376.f;
  return make_float2(re, im);
}

__device__ __forceinline__ uint32_t encode_code(float u) {
  int q = __float2int_rn(u);
  q = max(-32767, min(32767, q));
  return (uint32_t)(q + 32768);
}

__device__ __forceinline__ uint32_t encode_word(float re, float im, float inv) {
  return encode_code(__fmul_rn(re, inv)) | (encode_code(__fmul_rn(im, inv)) << 16);
}

// ------------------------------------------------------ colour-vector I/O
// Packed parity-half vectors (one per right-hand side; `S` = plane stride):
//   F64: double2 plane per colour; F32: float4 (c0, c1) + float2 (c2) planes;
//   I16: one uint4 per site = 3 code words + FP32 norm.

template <int PREC> struct SpinorIO;

template <> struct SpinorIO<PREC_F64> {
  using R = double;
  static __device__ __forceinline__ Vec3<double> load(const char *base, int S, int i) {
    const double2 *p = reinterpret_cast<const double2 *>(base);
    Vec3<double> v;
#pragma unroll
    for (int c = 0; c < 3; ++c) v.c[c] = __ldg(p + (size_t)c * S + i);
    return v;
  }
  static __device__ __forceinline__ void store(char *base, int S, int i, const Vec3<double> &v) {
    double2 *p = reinterpret_cast<double2 *>(base);
#pragma unroll
    for (int c = 0; c < 3; ++c) p[(size_t)c * S + i] = v.c[c];
  }
};

template <> struct SpinorIO<PREC_F32> {
  using R = float;
  static __device__ __forceinline__ Vec3<float> load(const char *base, int S, int i) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(base) + i);
    float2 b = __ldg(reinterpret_cast<const float2 *>(base + (size_t)16 * S) + i);
    Vec3<float> v;
    v.c[0] = make_float2(a.x, a.y);
    v.c[1] = make_float2(a.z, a.w);
    v.c[2] = b;
    return v;
  }
  static __device__ __forceinline__ void store(char *base, int S, int i, const Vec3<float> &v) {
    reinterpret_cast<float4 *>(base)[i] = make_float4(v.c[0].x, v.c[0].y, v.c[1].x, v.c[1].y);
    reinterpret_cast<float2 *>(base + (size_t)16 * S)[i] = v.c[2];
  }
};

template <> struct SpinorIO<PREC_I16> {
  using R = float;
  // values in code units together with the dequantisation factor n/32767
  static __device__ __forceinline__ Vec3<float> load_codes(const char *base, int i, float &scale) {
    uint4 w = __ldg(reinterpret_cast<const uint4 *>(base) + i);
    Vec3<float> v;
    v.c[0] = decode_word(w.x);
    v.c[1] = decode_word(w.y);
    v.c[2] = decode_word(w.z);
    scale = __uint_as_float(w.w) * (1.f / 32767.f);
    return v;
  }
  static __device__ __forceinline__ Vec3<float> load(const char *base, int S, int i) {
    float s;
    Vec3<float> v = load_codes(base, i, s);
#pragma unroll
    for (int c = 0; c < 3; ++c) { v.c[c].x *= s; v.c[c].y *= s; }
    return v;
  }
  // q = rint(v * (32767 / n)), n = max |v| over the six reals (FP32)
  static __device__ __forceinline__ void store(char *base, int S, int i, const Vec3<float> &v) {
    float n = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) n = fmaxf(n, fmaxf(fabsf(v.c[c].x), fabsf(v.c[c].y)));
    uint4 w;
    if (n > 0.f) {
      float inv = __fdiv_rn(32767.f, n);
      w.x = encode_word(v.c[0].x, v.c[0].y, inv);
      w.y = encode_word(v.c[1].x, v.c[1].y, inv);
      w.z = encode_word(v.c[2].x, v.c[2].y, inv);
    } else {
      w.x = w.y = w.z = 0x80008000u;
    }
    w.w = __float_as_uint(n);
    reinterpret_cast<uint4 *>(base)[i] = w;
  }
};

// FP64 <-> working precision conversions of whole colour vectors
template <typename RO, typename RI>
__device__ __forceinline__ Vec3<RO> convert(const Vec3<RI> &v) {
  Vec3<RO> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) { o.c[c].x = (RO)v.c[c].x; o.c[c].y = (RO)v.c[c].y; }
  return o;
}

// ------------------------------------------------------------ link layouts
// Per output parity and site, the 16 hop matrices of direction mu are, in
// order: F_mu(x), F_mu(x-mu)^dag (the "fat pair") and L_mu(x), L_mu(x-3mu)^dag
// (the "long pair").  Each site's bytes for direction mu are split into
// 16-byte planes (one plane = S consecutive 16-byte elements, one per site);
// a trailing 8-byte plane holds the remainder of 16-bit 18-real pairs.
//
//   precision/recon   fat pair          long pair
//   F64 / 18          18 x 16 B         18 x 16 B
//   F64 / 12          18 x 16 B         12 x 16 B (rows 0, 1 of each)
//   F32 / 18           9 x 16 B          9 x 16 B
//   F32 / 12           9 x 16 B          6 x 16 B
//   I16 / 18           4 x 16 B + 8 B    4 x 16 B + 8 B
//   I16 / 12           4 x 16 B + 8 B    3 x 16 B
//
// Direction blocks follow each other: mu = 0 fat, mu = 0 long, mu = 1 fat, ...

template <int PREC, int RECON> struct LinkLayout;

#define SQ_LAYOUT(P, RC, FAT16, FAT8, LONG16, LONG8)                              \
  template <> struct LinkLayout<P, RC> {                                          \
    static constexpr int fat16 = FAT16, fat8 = FAT8, long16 = LONG16, long8 = LONG8; \
    static constexpr int fat_bytes = 16 * FAT16 + 8 * FAT8;                       \
    static constexpr int long_bytes = 16 * LONG16 + 8 * LONG8;                    \
    static constexpr int mu_bytes = fat_bytes + long_bytes;                       \
    static constexpr int site_bytes = 4 * mu_bytes;                               \
  };
SQ_LAYOUT(PREC_F64, 18, 18, 0, 18, 0)
SQ_LAYOUT(PREC_F64, 12, 18, 0, 12, 0)
SQ_LAYOUT(PREC_F32, 18, 9, 0, 9, 0)
SQ_LAYOUT(PREC_F32, 12, 9, 0, 6, 0)
SQ_LAYOUT(PREC_I16, 18, 4, 1, 4, 1)
SQ_LAYOUT(PREC_I16, 12, 4, 1, 3, 0)
#undef SQ_LAYOUT

// Link scales handed to the kernels
struct LinkScales {
  float fat_k;      // I16: value = code * fat_k
  float long_k;     // I16: value = code * long_k
  float recon_f;    // 12-real: row2 = recon_f * conj(row0 x row1) in stored units
  double recon_d;   // same, FP64 kernels
  int keep;         // set in the kernel: links read again by a later tile
};

// Loader of the four hop matrices of direction mu at site i.
template <int PREC, int RECON> struct LinkIO;

template <int RECON> struct LinkIO<PREC_F64, RECON> {
  using LL = LinkLayout<PREC_F64, RECON>;
  // One pair of direction mu: the fat pair for KIND 0, the long pair for 1.
  template <int KIND>
  static __device__ __forceinline__ void load_pair(const char *links, int S, int i, int mu,
                                                   const LinkScales &ls, Mat3<double> m[2]) {
    const char *base = links + (size_t)mu * LL::mu_bytes * S;
    if (KIND == 1) base += (size_t)LL::fat_bytes * S;
    const uint64_t pol = l2_link_policy(ls.keep);
    constexpr int ne = (KIND == 0 || RECON == 18) ? 9 : 6;  // stored elements per matrix
#pragma unroll
    for (int k = 0; k < ne; ++k) {
      m[0].e[k] = ld_stream_d2(base + ((size_t)k * S + i) * 16, pol);
      m[1].e[k] = ld_stream_d2(base + ((size_t)(ne + k) * S + i) * 16, pol);
    }
    if constexpr (ne == 6) {
      reconstruct_row2(m[0], ls.recon_d);
      reconstruct_row2(m[1], ls.recon_d);
    }
  }
  static __device__ __forceinline__ void load(const char *links, int S, int i, int mu,
                                              const LinkScales &ls, Mat3<double> m[4]) {
    const char *fat = links + (size_t)mu * LL::mu_bytes * S;
    const char *lng = fat + (size_t)LL::fat_bytes * S;
    const uint64_t pol = l2_link_policy(ls.keep);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      m[0].e[k] = ld_stream_d2(fat + ((size_t)k * S + i) * 16, pol);
      m[1].e[k] = ld_stream_d2(fat + ((size_t)(9 + k) * S + i) * 16, pol);
    }
    constexpr int n = (RECON == 18) ? 9 : 6;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      m[2].e[k] = ld_stream_d2(lng + ((size_t)k * S + i) * 16, pol);
      m[3].e[k] = ld_stream_d2(lng + ((size_t)(n + k) * S + i) * 16, pol);
    }
    if (RECON == 12) {
      reconstruct_row2(m[2], ls.recon_d);
      reconstruct_row2(m[3], ls.recon_d);
    }
  }
};

__device__ __forceinline__ void f4_to_mats(const float4 *q, int nq, float *dst) {
  for (int k = 0; k < nq; ++k) {
    dst[4 * k + 0] = q[k].x; dst[4 * k + 1] = q[k].y;
    dst[4 * k + 2] = q[k].z; dst[4 * k + 3] = q[k].w;
  }
}

template <int RECON> struct LinkIO<PREC_F32, RECON> {
  using LL = LinkLayout<PREC_F32, RECON>;
  // One pair of direction mu: the fat pair (F_mu(x), F_mu(x-mu)^dag) for
  // kind 0, the long pair (L_mu(x), L_mu(x-3mu)^dag) for kind 1.
  template <int KIND>
  static __device__ __forceinline__ void load_pair(const char *links, int S, int i, int mu,
                                                   const LinkScales &ls, Mat3<float> m[2]) {
    const char *base = links + (size_t)mu * LL::mu_bytes * S;
    if (KIND == 1) base += (size_t)LL::fat_bytes * S;
    const uint64_t pol = l2_link_policy(ls.keep);
    constexpr int nq = (KIND == 0 || RECON == 18) ? 9 : 6;
    constexpr int ne = (KIND == 0 || RECON == 18) ? 9 : 6;  // stored elements per matrix
    float4 q[nq];
#pragma unroll
    for (int k = 0; k < nq; ++k) q[k] = ld_stream_f4(base + ((size_t)k * S + i) * 16, pol);
    float f[4 * nq];
#pragma unroll
    for (int k = 0; k < nq; ++k) {
      f[4 * k] = q[k].x; f[4 * k + 1] = q[k].y; f[4 * k + 2] = q[k].z; f[4 * k + 3] = q[k].w;
    }
#pragma unroll
    for (int e = 0; e < ne; ++e) {
      m[0].e[e] = make_float2(f[2 * e], f[2 * e + 1]);
      m[1].e[e] = make_float2(f[2 * ne + 2 * e], f[2 * ne + 2 * e + 1]);
    }
    if constexpr (ne == 6) {
      reconstruct_row2(m[0], ls.recon_f);
      reconstruct_row2(m[1], ls.recon_f);
    }
  }
  static __device__ __forceinline__ void load(const char *links, int S, int i, int mu,
                                              const LinkScales &ls, Mat3<float> m[4]) {
    const char *fat = links + (size_t)mu * LL::mu_bytes * S;
    const char *lng = fat + (size_t)LL::fat_bytes * S;
    const uint64_t pol = l2_link_policy(ls.keep);
    float4 q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) q[k] = ld_stream_f4(fat + ((size_t)k * S + i) * 16, pol);
    // floats 0..17 -> F_mu(x), 18..35 -> F_mu(x-mu)^dag
    float f[36];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      f[4 * k] = q[k].x; f[4 * k + 1] = q[k].y; f[4 * k + 2] = q[k].z; f[4 * k + 3] = q[k].w;
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      m[0].e[e] = make_float2(f[2 * e], f[2 * e + 1]);
      m[1].e[e] = make_float2(f[18 + 2 * e], f[18 + 2 * e + 1]);
    }
    if (RECON == 18) {
#pragma unroll
      for (int k = 0; k < 9; ++k) q[k] = ld_stream_f4(lng + ((size_t)k * S + i) * 16, pol);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        f[4 * k] = q[k].x; f[4 * k + 1] = q[k].y; f[4 * k + 2] = q[k].z; f[4 * k + 3] = q[k].w;
      }
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        m[2].e[e] = make_float2(f[2 * e], f[2 * e + 1]);
        m[3].e[e] = make_float2(f[18 + 2 * e], f[18 + 2 * e + 1]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) q[k] = ld_stream_f4(lng + ((size_t)k * S + i) * 16, pol);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        f[4 * k] = q[k].x; f[4 * k + 1] = q[k].y; f[4 * k + 2] = q[k].z; f[4 * k + 3] = q[k].w;
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        m[2].e[e] = make_float2(f[2 * e], f[2 * e + 1]);
        m[3].e[e] = make_float2(f[12 + 2 * e], f[12 + 2 * e + 1]);
      }
      reconstruct_row2(m[2], ls.recon_f);
      reconstruct_row2(m[3], ls.recon_f);
    }
  }
};

// 16-bit links: matrices come back in code units (value = code * k); the
// kernel applies k (fat_k / long_k) once per mat-vec result.
template <int RECON> struct LinkIO<PREC_I16, RECON> {
  using LL = LinkLayout<PREC_I16, RECON>;
  static __device__ __forceinline__ void load(const char *links, int S, int i, int mu,
                                              const LinkScales &ls, Mat3<float> m[4]) {
    const char *fat = links + (size_t)mu * LL::mu_bytes * S;
    const char *lng = fat + (size_t)LL::fat_bytes * S;
    const uint64_t pol = l2_link_policy(ls.keep);
    uint32_t w[18];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint4 q = ld_stream_u4(fat + ((size_t)k * S + i) * 16, pol);
      w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
    }
    {
      uint2 q = ld_stream_u2(fat + (size_t)64 * S + (size_t)i * 8, pol);
      w[16] = q.x; w[17] = q.y;
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      m[0].e[e] = decode_word(w[e]);
      m[1].e[e] = decode_word(w[9 + e]);
    }
    if (RECON == 18) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint4 q = ld_stream_u4(lng + ((size_t)k * S + i) * 16, pol);
        w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
      }
      uint2 q = ld_stream_u2(lng + (size_t)64 * S + (size_t)i * 8, pol);
      w[16] = q.x; w[17] = q.y;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        m[2].e[e] = decode_word(w[e]);
        m[3].e[e] = decode_word(w[9 + e]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint4 q = ld_stream_u4(lng + ((size_t)k * S + i) * 16, pol);
        w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        m[2].e[e] = decode_word(w[e]);
        m[3].e[e] = decode_word(w[6 + e]);
      }
      reconstruct_row2(m[2], ls.recon_f);
      reconstruct_row2(m[3], ls.recon_f);
    }
  }
};

// --------------------------------------------------------------- reductions
// Partial sums are formed per fixed chunk of CHUNK consecutive sites (warp
// shuffle tree, then the chunk's warps in order), so every sum is the same
// whatever block size a kernel is launched with.  The last block to finish
// adds the chunk partials in a fixed order.

constexpr int CHUNK = 128;
constexpr int WARPS_PER_CHUNK = CHUNK / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce NV values per thread over each chunk of the block; thread 0 of every
// chunk writes partial[v * chunk_stride + chunk] for v < nvalid,
// chunk_stride = number of chunks of the lattice (chunks past it belong to
// padding threads and are dropped).  smem needs NV * blockDim.x / 32 doubles.
template <int NV>
__device__ __forceinline__ void chunk_reduce(double (&val)[NV], double *smem, double *partial,
                                             int chunk_stride, int nvalid = NV) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int nwarps = blockDim.x >> 5;
  __syncthreads();  // smem may still be read by a previous call
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = warp_sum(val[v]);
    if (lane == 0) smem[v * nwarps + warp] = s;
  }
  __syncthreads();
  if ((threadIdx.x & (CHUNK - 1)) == 0) {
    int cfirst = warp;  // first warp of this chunk
    int chunk = (blockIdx.x * blockDim.x + threadIdx.x) / CHUNK;
    if (chunk < chunk_stride)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v >= nvalid) break;
      double s = 0;
#pragma unroll
      for (int w = 0; w < WARPS_PER_CHUNK; ++w) s += smem[v * nwarps + cfirst + w];
      partial[(size_t)v * chunk_stride + chunk] = s;
    }
  }
}

// Returns true in every thread of the block that finished last (of `total`
// blocks sharing `counter`); that block then sees all partials.  The ticket
// is one acquire-release atomic: release publishes this block's partials
// (made visible to thread 0 by the barrier), acquire makes every other
// block's partials visible to the last one -- no sequentially consistent
// device fence per block.
__device__ __forceinline__ bool last_block_arrived(unsigned *counter, unsigned total) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    unsigned ticket;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(ticket) : "l"(counter), "r"(1u) : "memory");
    is_last = (ticket == total - 1);
  }
  __syncthreads();
  return is_last;
}

// Barrier-free reduction over the sites of a grid row, in a fixed order.
// Every warp covers 32 consecutive sites (`site` is the calling thread's site
// index, consecutive across the lanes of a warp; blockDim a multiple of 32) and
// writes the shuffle-tree sum of its NV values as one partial per value.
// Warps are grouped 32 at a time by site index: the warp that arrives last in
// its group (one acquire-release ticket per group) adds the group's partials
// with a shuffle tree; the group that finishes last (a second ticket) adds
// the group sums, each lane over groups lane, lane + 32, ... in order, then a
// shuffle tree.  The order depends on site indices only, so every launch
// shape gives the same bits, and no block ever waits at a barrier.
//   inst[v]  base of value v's instance: nwchunks warp partials, then
//            ngroups group sums (red_stride doubles)
//   tickets  ngroups + 1 counters of this row (zero on entry; left zero)
// Returns true in every lane of the single warp that completed the sums;
// out[v] then holds sum v (all lanes).  All 32 lanes of each warp must call
// it together.  The values T are double, or float for the sloppy kernels:
// a warp's 32 sites are then summed in FP32 (GB300 issues FP64 at a small
// fraction of the FP32 rate, and a multi-system epilogue would otherwise
// spend more on its FP64 shuffle trees than on its loads), and every sum
// above the warp -- the accumulation over the lattice -- is in FP64.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

template <int NV, typename T>
__device__ __forceinline__ bool warp_tree_reduce(const T (&val)[NV], int nvalid,
                                                 double *const (&inst)[NV], const Geom &g,
                                                 int site, unsigned *tickets,
                                                 double (&out)[NV]) {
  const int lane = threadIdx.x & 31;
  const int wc = site >> 5;
  if (wc >= g.nwchunks) return false;  // a warp wholly past the last site
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T sv = warp_sum(val[v]);
    if (lane == 0 && v < nvalid) inst[v][wc] = (double)sv;
  }
  const int grp = wc >> 5;
  const int in_grp = min(32, g.nwchunks - grp * 32);
  unsigned t = 0;
  if (lane == 0) t = atom_add_acq_rel(tickets + grp, 1u);
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t != (unsigned)(in_grp - 1)) return false;
  __syncwarp();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v >= nvalid) break;
    const double x = (lane < in_grp) ? __ldcg(inst[v] + grp * 32 + lane) : 0.0;
    const double gs = warp_sum(x);
    if (lane == 0) inst[v][g.nwchunks + grp] = gs;
  }
  if (lane == 0) {
    tickets[grp] = 0;
    t = atom_add_acq_rel(tickets + g.ngroups, 1u);
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t != (unsigned)(g.ngroups - 1)) return false;
  __syncwarp();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    out[v] = 0.0;
    if (v >= nvalid) continue;
    double acc = 0.0;
    for (int k = lane; k < g.ngroups; k += 32) acc += __ldcg(inst[v] + g.nwchunks + k);
    out[v] = warp_sum(acc);
  }
  if (lane == 0) tickets[g.ngroups] = 0;
  return true;
}

// First half of warp_tree_reduce alone: every warp stores the shuffle-tree
// sum of its 32 sites' values as one partial per value (inst[v][site / 32])
// and goes on; a separate kernel adds the partials (cg_finish_kernel).  No
// warp waits for a ticket, and the Dslash kernel's last warp has no serial
// sum to run before the next kernel may start.
template <int NV, typename T>
__device__ __forceinline__ void warp_partials(const T (&val)[NV], int nvalid,
                                              double *const (&inst)[NV], const Geom &g,
                                              int site) {
  const int lane = threadIdx.x & 31;
  const int wc = site >> 5;
  if (wc >= g.nwchunks) return;  // a warp wholly past the last site
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T sv = warp_sum(val[v]);
    if (lane == 0 && v < nvalid) inst[v][wc] = (double)sv;
  }
}

// Fixed-order sum of n partials by a block of exactly WIDE_SUM_THREADS
// threads: thread t adds elements t, t + W, t + 2W, ... in order (eight
// loads in flight at a time), then a shuffle tree per warp and the warps'
// sums in order.  The order depends on n only.  All threads of the block
// call it; the result is valid in thread 0.
constexpr int WIDE_SUM_THREADS = 1024;

__device__ __forceinline__ double block_sum_wide(const double *p, int n, double *smem) {
  constexpr int W = WIDE_SUM_THREADS;
  double s = 0;
  for (int k0 = threadIdx.x; k0 < n; k0 += 8 * W) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u * W;
      v[u] = (k < n) ? __ldcg(p + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = s;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < W / 32; ++w) t += smem[w];
  return t;
}

// Fixed-order sum of n partials: 128 virtual lanes (the block's first 128
// threads) accumulate strided elements in order k, k + 128, k + 256, ...,
// then a fixed shuffle tree and the four warp sums in order.  Independent of
// the block size, so every configuration gives the same bits.  All threads
// of the block call it; the result is valid in every thread.
constexpr int SUM_LANES = 128;

__device__ __forceinline__ double block_sum_fixed(const double *p, int n, double *smem) {
  double s = 0;
  if (threadIdx.x < SUM_LANES) {
    for (int k0 = threadIdx.x; k0 < n; k0 += 8 * SUM_LANES) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {  // eight loads in flight per round
        int k = k0 + u * SUM_LANES;
        v[u] = (k < n) ? __ldcg(p + k) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
  }
  s = warp_sum(s);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0 && warp < SUM_LANES / 32) smem[warp] = s;
  __syncthreads();
  double t = 0;
#pragma unroll
  for (int w = 0; w < SUM_LANES / 32; ++w) t += smem[w];
  __syncthreads();
  return t;
}

}  // namespace sq
