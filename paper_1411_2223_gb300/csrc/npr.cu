// The one-colour four-fermion operator of the NPR code in Sec. 2 (Eq. 1,
// Fig. 2, Table 3), in FP64 on the GPU.
//
// For every hypercube z of the lattice (corner sites z_A = 2z + A, A in
// {0,1}^4, A = A_x + 2 A_y + 4 A_z + 8 A_t) and every operator
// (S1, F1, S2, F2):
//   O[a1][a2][a3][a4](z) = sum_{A,C} M1[A][B] M2[C][D]
//       (G1(z_A)^dag U_AD G4(z_D))[a1][a4] (G3(z_C)^dag U_CB G2(z_B))[a3][a2]
// with B = A ^ S1 ^ F1 and D = C ^ S2 ^ F2: the hypercube spin-taste matrix
// (gamma_S x xi_F)_{AB} = Tr(gamma_A^dag gamma_S gamma_B gamma_F^dag) / 4 has
// one entry, +1 or -1, per row, at B = A ^ S ^ F (spin_taste_sign below).
// U_AD(z) is the mean of the link products over the shortest paths from z_A
// to z_D.  The propagators G^f are [site][colour][source colour]; flavours 1
// and 3 enter conjugated, as the antiquark fields of Eq. 1.
//
// One CTA works on one hypercube at a time (persistent grid, one CTA of 512
// threads per SM), in shared memory:
//   1. the 16 corners' propagators and the 32 links inside the hypercube
//      arrive by cp.async, prefetched while the previous hypercube's
//      contraction runs;
//   2. U_AD for A < D, level by level in the distance n = |A ^ D|, from
//      U_AD = (1/n) sum_{mu in A ^ D} U_{A, A^mu} U_{A^mu, D}: a shortest
//      path starts with any of the n differing directions, each first in
//      (n-1)! of the n! paths.  U_DA = U_AD^dag is read, not stored;
//   3. P[A][D] = G1(A)^dag U_AD G4(D) and Q[C][B] = G3(C)^dag U_CB G2(B) for
//      all 256 corner pairs, shared by every operator;
//   4. per operator and output, the 256-term sum over (A, C) of
//      +-P[A][C ^ t2][a1][a4] Q[C][A ^ t1][a3][a2], t = S ^ F, with three real
//      multiply-adds per complex term (contract below).
// All of it is FP64 arithmetic (about 1.6 MFLOP per hypercube for 8
// operators, counting 8 per complex multiply-add, against 14 KB of input), so
// the kernel is bound by the FP64 units, not by HBM.  Per-hypercube results are written when asked for; the
// sums over hypercubes go through per-CTA partials and a fixed-order second
// pass, so they do not depend on scheduling.
#include <cmath>
#include <cstdint>

#include "sq_host.h"

namespace sq {
namespace {

int spin_taste_sign(int s, int f, int a) {
  // gamma_X gamma_Y = sigma(X, Y) gamma_{X^Y}: each gamma_j of Y moves left
  // past the gamma_i of X with i > j.  gamma_X^dag = (-1)^(n(n-1)/2) gamma_X
  // for |X| = n.  With B = A ^ S ^ F,
  //   gamma_A^dag gamma_S gamma_B gamma_F^dag
  //     = r(A) r(F) sigma(A, S) sigma(A^S, B) sigma(F, F) * 1
  // and sigma(F, F) = r(F).
  auto sigma = [](int x, int y) {
    int n = 0;
    for (int i = 0; i < 4; ++i)
      if ((x >> i) & 1)
        for (int j = 0; j < i; ++j) n += (y >> j) & 1;
    return (n & 1) ? -1 : 1;
  };
  auto rev = [](int x) {
    const int n = __builtin_popcount(x);
    return ((n * (n - 1) / 2) & 1) ? -1 : 1;
  };
  const int b = a ^ s ^ f;
  return rev(a) * sigma(a, s) * sigma(a ^ s, b);
}

constexpr int kThreads = 512;
constexpr int kMaxOps = SQ_NPR_MAX_OPS;
constexpr int kItemsPerThread = (kMaxOps * 81 + kThreads - 1) / kThreads;
constexpr int kTri = 136;                  // corner pairs A <= D
constexpr int kLoadChunks = 4 * 16 * 9 + 32 * 9;
constexpr size_t kSmemBytes =
    sizeof(double2) * (kTri * 9 + 4 * 16 * 9 + 2 * 256 * 9) + sizeof(double) * 2 * 256 * 9;

struct NprOp {
  uint16_t neg1, neg2;  // bit A (C): the entry of row A (C) is -1
  uint8_t t1, t2;       // S1 ^ F1, S2 ^ F2
};

struct NprArgs {
  const double2 *links;    // [site][mu][3][3]
  const double2 *prop[4];  // [site][3][3]
  double2 *out_hc;         // this group's first op of [hypercube][op][81], or null
  long hc_stride;          // elements per hypercube of out_hc (all ops x 81)
  double2 *partial;        // [cta][op][81]
  int H[4];                // hypercubes per direction
  long st[4];              // site strides
  int nhc;
  int nops;
  NprOp ops[kMaxOps];
};

__device__ __forceinline__ int tri(int a, int d) {  // a <= d
  return 16 * a - (a * (a - 1)) / 2 + (d - a);
}

__device__ __forceinline__ double flip(double v, unsigned neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)neg << 63));
}

// element (i, j) of U_XY for any corners X, Y
__device__ __forceinline__ double2 u_elem(const double2 *ut, int x, int y, int i, int j) {
  const bool sw = x > y;
  const int lo = sw ? y : x, hi = sw ? x : y;
  const double2 v = ut[tri(lo, hi) * 9 + (sw ? 3 * j + i : 3 * i + j)];
  return make_double2(v.x, flip(v.y, sw));
}

__device__ __forceinline__ void cmac(double2 &c, double2 a, double2 b) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
}

__device__ __forceinline__ void cmac_conj(double2 &c, double2 a, double2 b) {  // conj(a) b
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Step 1: propagators of the 16 corners and links inside hypercube h.
__device__ void issue_loads(const NprArgs &a, int h, double2 *gs, double2 *ut) {
  int r = h;
  long s0 = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    s0 += 2L * (r % a.H[mu]) * a.st[mu];
    r /= a.H[mu];
  }
  for (int i = threadIdx.x; i < kLoadChunks; i += kThreads) {
    const double2 *src;
    double2 *dst;
    if (i < 4 * 16 * 9) {
      const int f = i / 144, c = (i / 9) % 16, e = i % 9;
      const long site = s0 + (c & 1) * a.st[0] + ((c >> 1) & 1) * a.st[1] +
                        ((c >> 2) & 1) * a.st[2] + (c >> 3) * a.st[3];
      src = a.prop[f] + site * 9 + e;
      dst = gs + (f * 16 + c) * 9 + e;
    } else {
      const int j = i - 4 * 16 * 9;
      const int mu = j / 72, k = (j / 9) % 8, e = j % 9;
      const int c = ((k >> mu) << (mu + 1)) | (k & ((1 << mu) - 1));  // corner with bit mu = 0
      const long site = s0 + (c & 1) * a.st[0] + ((c >> 1) & 1) * a.st[1] +
                        ((c >> 2) & 1) * a.st[2] + (c >> 3) * a.st[3];
      src = a.links + (site * 4 + mu) * 9 + e;
      dst = ut + tri(c, c | (1 << mu)) * 9 + e;
    }
    cp_async16(dst, src);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Step 2, distance n: U_AD for the 8 C(4, n) pairs A < D with |A ^ D| = n.
__device__ void path_level(double2 *ut, int n) {
  const int npairs = n == 2 ? 48 : (n == 3 ? 32 : 8);
  const double inv = n == 2 ? 0.5 : (n == 3 ? 1.0 / 3.0 : 0.25);
  for (int it = threadIdx.x; it < npairs * 9; it += kThreads) {
    const int k = it / 9, e = it % 9, i = e / 3, j = e % 3;
    int x = 0;  // the (k/8)-th difference mask with n bits
    for (int m = 1, seen = 0; m < 16; ++m)
      if (__popc(m) == n && seen++ == (k >> 3)) {
        x = m;
        break;
      }
    const int top = 31 - __clz(x);
    const int lo = k & 7;
    const int A = ((lo >> top) << (top + 1)) | (lo & ((1 << top) - 1));  // bit top = 0
    const int D = A ^ x;
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      if (!((x >> mu) & 1)) continue;
      const int m = A ^ (1 << mu);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) cmac(s, u_elem(ut, A, m, i, kk), u_elem(ut, m, D, kk, j));
    }
    ut[tri(A, D) * 9 + e] = make_double2(s.x * inv, s.y * inv);
  }
}

// Step 3: P[X][Y] = G1(X)^dag U_XY G4(Y) and Q[X][Y] = G3(X)^dag U_XY G2(Y),
// one column of one pair per item.
__device__ void sandwiches(const double2 *ut, const double2 *gs, double2 *ps, double2 *qs,
                           double *pss, double *qss) {
  for (int it = threadIdx.x; it < 2 * 256 * 3; it += kThreads) {
    const int which = it >= 768;
    const int rem = it - which * 768;
    const int pair = rem / 3, col = rem % 3;
    const int x = pair >> 4, y = pair & 15;
    const double2 *gl = gs + ((which ? 2 : 0) * 16 + x) * 9;
    const double2 *gr = gs + ((which ? 1 : 3) * 16 + y) * 9;
    double2 h[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h[c] = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(h[c], u_elem(ut, x, y, c, k), gr[3 * k + col]);
    }
    double2 *dst = (which ? qs : ps) + pair * 9;
    double *dsum = (which ? qss : pss) + pair * 9;
#pragma unroll
    for (int a1 = 0; a1 < 3; ++a1) {
      double2 v = make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < 3; ++c) cmac_conj(v, gl[3 * c + a1], h[c]);
      dst[3 * a1 + col] = v;
      dsum[3 * a1 + col] = v.x + v.y;
    }
  }
}

// Step 4: output o = 27 a1 + 9 a2 + 3 a3 + a4 of one operator.  The complex
// products go by the 3M method (Higham, "Stability of a method for
// multiplying complex matrices with three real matrix multiplications",
// SIMAX 1992): with re + im of P and Q stored beside them,
//   sum p q = (T1 - T2) + i (T3 - T1 - T2),
//   T1 = sum p.re q.re,  T2 = sum p.im q.im,  T3 = sum (p.re + p.im)(q.re + q.im),
// three real multiply-adds per term instead of four.
__device__ __forceinline__ double2 contract(const double2 *ps, const double2 *qs,
                                            const double *pss, const double *qss, NprOp op,
                                            int o) {
  const int a1 = o / 27, a2 = (o / 9) % 3, a3 = (o / 3) % 3, a4 = o % 3;
  const int pe = 3 * a1 + a4, qe = 3 * a3 + a2;
  double t1[4], t2[4], t3[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) t1[k] = t2[k] = t3[k] = 0.0;
#pragma unroll 2
  for (int A = 0; A < 16; ++A) {
    const int qo = (A ^ op.t1) * 9 + qe;  // Q[C][A ^ t1] at qo + C * 16 * 9
    const int po = A * 16 * 9 + pe;       // P[A][D] at po + D * 9
    const unsigned sa = (op.neg1 >> A) & 1;
#pragma unroll
    for (int C = 0; C < 16; ++C) {
      const int pi = po + (C ^ op.t2) * 9, qi = qo + C * 16 * 9;
      const double2 p = ps[pi], q = qs[qi];
      const double sp = pss[pi], sq = qss[qi];
      const unsigned neg = sa ^ ((op.neg2 >> C) & 1);
      t1[C & 3] = fma(flip(p.x, neg), q.x, t1[C & 3]);
      t2[C & 3] = fma(flip(p.y, neg), q.y, t2[C & 3]);
      t3[C & 3] = fma(flip(sp, neg), sq, t3[C & 3]);
    }
  }
  const double T1 = (t1[0] + t1[1]) + (t1[2] + t1[3]);
  const double T2 = (t2[0] + t2[1]) + (t2[2] + t2[3]);
  const double T3 = (t3[0] + t3[1]) + (t3[2] + t3[3]);
  return make_double2(T1 - T2, (T3 - T1) - T2);
}

__global__ void __launch_bounds__(kThreads, 1) npr_kernel(const NprArgs a) {
  extern __shared__ double2 smem[];
  double2 *ut = smem;              // [pair A <= D][3][3]
  double2 *gs = ut + kTri * 9;     // [flavour][corner][3][3]
  double2 *ps = gs + 4 * 16 * 9;   // [A][D][a1][a4]
  double2 *qs = ps + 256 * 9;      // [C][B][a3][a2]
  double *pss = reinterpret_cast<double *>(qs + 256 * 9);  // re + im of ps
  double *qss = pss + 256 * 9;                             // re + im of qs
  const int tid = threadIdx.x;
  for (int i = tid; i < 16 * 9; i += kThreads) {
    const int c = i / 9, e = i % 9;
    ut[tri(c, c) * 9 + e] = make_double2(e % 4 == 0 ? 1.0 : 0.0, 0.0);
  }
  const int nitems = a.nops * 81;
  double2 tot[kItemsPerThread];
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) tot[r] = make_double2(0.0, 0.0);
  int h = blockIdx.x;
  if (h < a.nhc) issue_loads(a, h, gs, ut);
  for (; h < a.nhc; h += gridDim.x) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    for (int n = 2; n <= 4; ++n) {
      path_level(ut, n);
      __syncthreads();
    }
    sandwiches(ut, gs, ps, qs, pss, qss);
    __syncthreads();
    if (h + (int)gridDim.x < a.nhc) issue_loads(a, h + gridDim.x, gs, ut);
#pragma unroll
    for (int r = 0; r < kItemsPerThread; ++r) {
      const int it = tid + r * kThreads;
      if (it < nitems) {
        const double2 v = contract(ps, qs, pss, qss, a.ops[it / 81], it % 81);
        if (a.out_hc) a.out_hc[(long)h * a.hc_stride + it] = v;
        tot[r].x += v.x;
        tot[r].y += v.y;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    const int it = tid + r * kThreads;
    if (it < nitems) a.partial[(long)blockIdx.x * nitems + it] = tot[r];
  }
}

// Sum of the per-CTA partials, CTA 0 first.
__global__ void npr_sum_kernel(const double2 *partial, int nparts, int n, double2 *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nparts; ++b) {
    const double2 v = partial[(long)b * n + i];
    s.x += v.x;
    s.y += v.y;
  }
  out[i] = s;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace sq

using namespace sq;

extern "C" int sq_spin_taste(int s, int f, int partner[16], int sign[16]) {
  if (s < 0 || s > 15 || f < 0 || f > 15 || !partner || !sign) return SQ_ERR_ARG;
  for (int a = 0; a < 16; ++a) {
    partner[a] = a ^ s ^ f;
    sign[a] = spin_taste_sign(s, f, a);
  }
  return SQ_OK;
}

extern "C" int npr_four_fermion(sq_ctx *ctx, const int dims[4], const double *links_dev,
                                const double *const props_dev[4], int nops, const int *ops,
                                double *out_dev, double *out_hc_dev, void *stream) {
  if (!ctx || !dims || !links_dev || !props_dev || nops < 0 || nops > (1 << 20))
    return SQ_ERR_ARG;
  if (nops > 0 && (!ops || !out_dev)) return SQ_ERR_ARG;
  long vol;
  int rc = check_lattice_dims(dims, &vol);
  if (rc) return rc;
  if (!aligned16(links_dev) || !aligned16(out_dev) || !aligned16(out_hc_dev)) return SQ_ERR_ARG;
  for (int f = 0; f < 4; ++f)
    if (!props_dev[f] || !aligned16(props_dev[f])) return SQ_ERR_ARG;
  for (long k = 0; k < 4L * nops; ++k)
    if (ops[k] < 0 || ops[k] > 15) return SQ_ERR_ARG;
  if (nops == 0) return SQ_OK;

  NprArgs a{};
  a.links = reinterpret_cast<const double2 *>(links_dev);
  for (int f = 0; f < 4; ++f) a.prop[f] = reinterpret_cast<const double2 *>(props_dev[f]);
  a.nhc = (int)(vol / 16);
  for (int mu = 0; mu < 4; ++mu) a.H[mu] = dims[mu] / 2;
  a.st[0] = 1;
  for (int mu = 1; mu < 4; ++mu) a.st[mu] = a.st[mu - 1] * dims[mu - 1];
  a.hc_stride = 81L * nops;

  cudaSetDevice(ctx->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamLegacy;  // NULL: default stream
  SQ_CUDA_TRY(cudaFuncSetAttribute(npr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kSmemBytes));
  int per_sm = 0, sms = 0;
  SQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, npr_kernel, kThreads,
                                                            kSmemBytes));
  SQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  if (per_sm < 1) per_sm = 1;
  const int grid = (int)std::min<long>(a.nhc, (long)per_sm * sms);
  void *partial = nullptr;
  SQ_CUDA_TRY(cudaMallocAsync(&partial, sizeof(double2) * (size_t)grid * kMaxOps * 81, st));
  a.partial = static_cast<double2 *>(partial);
  cudaError_t e = cudaSuccess;
  // kMaxOps operators per launch pair; each group recomputes the averaged
  // links and the sandwiches P, Q of every hypercube
  for (int g0 = 0; g0 < nops && e == cudaSuccess; g0 += kMaxOps) {
    a.nops = std::min(kMaxOps, nops - g0);
    for (int k = 0; k < a.nops; ++k) {
      const int *o = ops + 4 * (g0 + k);
      NprOp &p = a.ops[k];
      p.t1 = (uint8_t)(o[0] ^ o[1]);
      p.t2 = (uint8_t)(o[2] ^ o[3]);
      p.neg1 = p.neg2 = 0;
      for (int c = 0; c < 16; ++c) {
        if (spin_taste_sign(o[0], o[1], c) < 0) p.neg1 |= (uint16_t)(1u << c);
        if (spin_taste_sign(o[2], o[3], c) < 0) p.neg2 |= (uint16_t)(1u << c);
      }
    }
    a.out_hc = out_hc_dev ? reinterpret_cast<double2 *>(out_hc_dev) + 81L * g0 : nullptr;
    const int nitems = a.nops * 81;
    npr_kernel<<<grid, kThreads, kSmemBytes, st>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      npr_sum_kernel<<<(nitems + 255) / 256, 256, 0, st>>>(
          a.partial, grid, nitems, reinterpret_cast<double2 *>(out_dev) + 81L * g0);
      e = cudaGetLastError();
      ctx->launches += 2;
    }
  }
  cudaFreeAsync(partial, st);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "npr kernels", __FILE__, __LINE__);
    return SQ_ERR_CUDA;
  }
  return SQ_OK;
}
