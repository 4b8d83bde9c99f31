// The asqtad even-odd Dslash kernel family.
//
//   (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu) - F_mu(x-mu)^dag psi(x-mu)
//                                      + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^dag psi(x-3mu) ]
//
// for the output sites x of one parity (the paper's CG inverter on the asqtad
// lattice, Sec. 2 / Fig. 1, spends its time in this operator).  One thread
// per output site; each thread reads the site's 16 hop matrices once (16-byte
// streaming loads, site-major planes) and applies them to NR right-hand
// sides.  The neighbours' colour vectors are gathered through L1/L2 (the
// input field of one parity is small enough to stay in L2).
//
// Epilogues:
//   MODE_PLAIN  out = D in
//   MODE_MDAGM  out = m^2 p - D in               (second Dslash of A = m^2 - D_eo D_oe)
//               + per-chunk partials of Re<p, out>, and the last block sets
//               alpha = rr / <p, Ap> for every running system
//   MODE_RESID  r = b - (m^2 x - D in), FP64     (reliable update: true residual)
//               with x = x64 + xs folded into x64 first; r is written in the
//               sloppy precision OUTP, + partials of |r|^2 and <r, p_sloppy>;
//               the last block finishes the update
//   MODE_NORM   out = D in (the CG's D_oe p), + per-warp partials of
//               |out|^2 + m^2 |in|^2 over the own index: that is
//               <p, A p> = |M p|^2 for A = M^dag M restricted to the even
//               sites, since D_eo = -D_oe^dag; the finish kernel that
//               follows adds them and sets alpha
//   MODE_UPDATE Ap = m^2 p - D in, not stored: xs += alpha p, r -= alpha Ap
//               (r is `out`), + per-warp partials of |r|^2; the finish
//               kernel that follows adds them and takes the CG step (beta,
//               or a reliable-update request)
// For a reliable update the PLAIN FP64 kernel gathers x64 + xs (the FP64
// solution plus its sloppy increment since the previous update).
#pragma once

#include "sq_device.cuh"
#include "cg_finish.cuh"

namespace sq {

enum DslashMode { MODE_PLAIN = 0, MODE_MDAGM = 1, MODE_RESID = 2, MODE_NORM = 3, MODE_UPDATE = 4 };
enum Gate { GATE_NONE = 0, GATE_RUNNING = 1, GATE_RU = 2 };

struct DslashArgs {
  Geom g;
  int out_parity;
  const char *links;          // link planes of the output parity (this precision/recon)
  LinkScales ls;
  const char *in;             // nrhs input fields (parity 1 - out_parity)
  char *out;                  // nrhs output fields
  size_t in_fb, out_fb;       // bytes between consecutive rhs fields
  int nrhs;
  double m2_const;            // MDAGM without slots: the mass^2
  // MDAGM: p (output parity, same precision as in)
  const char *p;
  size_t p_fb;
  // RESID: FP64 x and b, sloppy p
  const char *x64, *b64;
  size_t f64_fb;
  // reliable update: solution increment xs (precision xs_prec) added to the
  // FP64 input at every gathered neighbour (PLAIN) or folded into x64 (RESID)
  char *xs;
  size_t xs_fb;
  int xs_prec;
  const char *ps;
  size_t ps_fb;
  SlotState *slots;           // nullptr: no CG state (operator application only)
  ShiftState *shifts;         // multi-shift CG: shifted systems updated with alpha
  int nshift;
  double *partial;            // [value][rhs][chunk]
  unsigned *counter;
  int gate;
  int max_grid;               // > 0: the reliable-update pair's FP64 kernels (PLAIN, RESID)
                              // run as dslash_gated_kernel on at most this many blocks
};

template <int PREC> struct AccumType { using R = float; };
template <> struct AccumType<PREC_F64> { using R = double; };

__device__ __forceinline__ bool slot_active(const SlotState *s, int gate) {
  if (gate == GATE_RUNNING) return s->status == SLOT_RUNNING;
  if (gate == GATE_RU) return s->ru_pending != 0;
  return true;
}

// Colour vector of hop neighbour n for rhs field `f`, multiplied by `scale`
// (boundary sign, and for 16-bit data the code scales).
template <int PREC, typename R>
__device__ __forceinline__ Vec3<R> gather(const char *f, int S, int n, float scale) {
  if constexpr (PREC == PREC_I16) {
    float s;
    Vec3<float> v = SpinorIO<PREC_I16>::load_codes(f, n, s);
    s *= scale;
#pragma unroll
    for (int c = 0; c < 3; ++c) { v.c[c].x *= s; v.c[c].y *= s; }
    return v;
  } else {
    Vec3<R> v = SpinorIO<PREC>::load(f, S, n);
    if (scale < 0.f) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { v.c[c].x = -v.c[c].x; v.c[c].y = -v.c[c].y; }
    }
    return v;
  }
}

// Neighbour input of the Dslash: the field itself, or for the FP64 operator
// of a reliable update the FP64 solution plus its sloppy increment.
template <int PREC, int MODE, typename R>
__device__ __forceinline__ Vec3<R> gather_in(const char *f, const char *fx, int xs_prec, int S,
                                             int n, float scale) {
  if constexpr (PREC == PREC_F64 && MODE == 0) {
    if (fx != nullptr) {
      Vec3<double> v = SpinorIO<PREC_F64>::load(f, S, n);
      if (xs_prec == PREC_F32) {
        Vec3<float> d = SpinorIO<PREC_F32>::load(fx, S, n);
#pragma unroll
        for (int c = 0; c < 3; ++c) { v.c[c].x += (double)d.c[c].x; v.c[c].y += (double)d.c[c].y; }
      } else {
        Vec3<double> d = SpinorIO<PREC_F64>::load(fx, S, n);
#pragma unroll
        for (int c = 0; c < 3; ++c) { v.c[c].x += d.c[c].x; v.c[c].y += d.c[c].y; }
      }
      if (scale < 0.f) {
#pragma unroll
        for (int c = 0; c < 3; ++c) { v.c[c].x = -v.c[c].x; v.c[c].y = -v.c[c].y; }
      }
      return v;
    }
  }
  return gather<PREC, R>(f, S, n, scale);
}

// acc -= M v
template <typename R>
__device__ __forceinline__ void mat_vec_sub(Vec3<R> &acc, const Mat3<R> &m, const Vec3<R> &v) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc.c[r].x = fma(-m.e[3 * r + c].x, v.c[c].x, acc.c[r].x);
      acc.c[r].x = fma(m.e[3 * r + c].y, v.c[c].y, acc.c[r].x);
      acc.c[r].y = fma(-m.e[3 * r + c].x, v.c[c].y, acc.c[r].y);
      acc.c[r].y = fma(-m.e[3 * r + c].y, v.c[c].x, acc.c[r].y);
    }
  }
}

// ------------------------------------------------------------ 16-bit body
// 16-bit links stay in their packed words until the mat-vec that uses them
// (half the registers of decoded floats), which leaves room to load the words
// of direction mu+1 while direction mu is computed: every thread keeps one
// direction of links in flight through its whole life instead of waiting for
// each direction in turn.  Every hop's sign (eta, backward hop, antiperiodic
// wrap) and scale (link code scale, neighbour norm) is folded into one factor
// applied to the neighbour vector, so all 16 products accumulate directly.

template <int RECON> struct I16Words {
  static constexpr int NL = (RECON == 18) ? 18 : 12;
  uint32_t w[18 + NL];  // fat pair (9 + 9 words), long pair (9 + 9, or 6 + 6)
};

__device__ __forceinline__ void put4(uint32_t *w, uint4 q) {
  w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
}

template <int RECON>
__device__ __forceinline__ void i16_load_words(const char *links, int S, int i, int mu,
                                               I16Words<RECON> &d, bool keep) {
  using LL = LinkLayout<PREC_I16, RECON>;
  const char *fat = links + (size_t)mu * LL::mu_bytes * S;
  const char *lng = fat + (size_t)LL::fat_bytes * S;
  const uint64_t pol = l2_link_policy(keep);
#pragma unroll
  for (int k = 0; k < 4; ++k) put4(d.w + 4 * k, ld_stream_u4(fat + ((size_t)k * S + i) * 16, pol));
  {
    uint2 q = ld_stream_u2(fat + (size_t)64 * S + (size_t)i * 8, pol);
    d.w[16] = q.x; d.w[17] = q.y;
  }
  if constexpr (RECON == 18) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      put4(d.w + 18 + 4 * k, ld_stream_u4(lng + ((size_t)k * S + i) * 16, pol));
    uint2 q = ld_stream_u2(lng + (size_t)64 * S + (size_t)i * 8, pol);
    d.w[34] = q.x; d.w[35] = q.y;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      put4(d.w + 18 + 4 * k, ld_stream_u4(lng + ((size_t)k * S + i) * 16, pol));
  }
}

// acc += M v, M given as 9 code words (row-major)
__device__ __forceinline__ void mat_vec_words(Vec3<float> &acc, const uint32_t *w,
                                              const Vec3<float> &v) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 m = decode_word(w[3 * r + c]);
      acc.c[r].x = fma(m.x, v.c[c].x, acc.c[r].x);
      acc.c[r].x = fma(-m.y, v.c[c].y, acc.c[r].x);
      acc.c[r].y = fma(m.x, v.c[c].y, acc.c[r].y);
      acc.c[r].y = fma(m.y, v.c[c].x, acc.c[r].y);
    }
  }
}

// Neighbour colour vector in code units times (site norm / 32767) * f.
__device__ __forceinline__ Vec3<float> i16_vector(const uint4 q, float f) {
  const float s = __uint_as_float(q.w) * (1.f / 32767.f) * f;
  Vec3<float> v;
  v.c[0] = decode_word(q.x);
  v.c[1] = decode_word(q.y);
  v.c[2] = decode_word(q.z);
#pragma unroll
  for (int c = 0; c < 3; ++c) { v.c[c].x *= s; v.c[c].y *= s; }
  return v;
}

// buf holds direction 0's words on entry (loaded by the caller before the
// kernel waited for its predecessor); each later direction's words are
// loaded at its top.  Measured against keeping the next direction's words
// in flight: holding one direction needs ~80 registers instead of ~128, the
// 24 resident warps per SM this allows hide more latency than the prefetch
// did (20^3 x 64: 23.4 vs 27.0 us; 32^3 x 64: 83.6 vs 94.2 us, 12-real).
template <int RECON, int NR>
__device__ __forceinline__ void i16_hops(const DslashArgs &a, const LinkScales &ls,
                                         const SiteCoords &sc, int i, int r0,
                                         const bool (&active)[NR], Vec3<float> (&acc)[NR],
                                         I16Words<RECON> &buf) {
  const Geom &g = a.g;
  const int S = g.stride;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (mu > 0) i16_load_words<RECON>(a.links, S, i, mu, buf, ls.keep);
    const uint32_t *w = buf.w;
    int nb[4];
    float f[4];
    nb[0] = hop<+1>(g, sc, mu, f[0]);
    nb[1] = hop<-1>(g, sc, mu, f[1]);
    nb[2] = hop<+3>(g, sc, mu, f[2]);
    nb[3] = hop<-3>(g, sc, mu, f[3]);
    const float eta = eta_sign(sc, mu);
    const float kf = eta * ls.fat_k, kl = eta * ls.long_k;
    f[0] *= kf;
    f[1] *= -kf;
    f[2] *= kl;
    f[3] *= -kl;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (!active[r]) continue;
      const uint4 *in = reinterpret_cast<const uint4 *>(a.in + (size_t)(r0 + r) * a.in_fb);
      uint4 q[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) q[h] = __ldg(in + nb[h]);
      mat_vec_words(acc[r], w, i16_vector(q[0], f[0]));
      mat_vec_words(acc[r], w + 9, i16_vector(q[1], f[1]));
      if constexpr (RECON == 18) {
        mat_vec_words(acc[r], w + 18, i16_vector(q[2], f[2]));
        mat_vec_words(acc[r], w + 27, i16_vector(q[3], f[3]));
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          Mat3<float> m;
#pragma unroll
          for (int e = 0; e < 6; ++e) m.e[e] = decode_word(w[18 + 6 * h + e]);
          reconstruct_row2(m, ls.recon_f);
          mat_vec_acc(acc[r], m, i16_vector(q[2 + h], f[2 + h]));
        }
      }
    }
  }
}

// ------------------------------------------------------ pair at a time
// One pair of hop matrices (fat or long) is held at a time, with the hop's
// sign (eta, backward hop, antiperiodic wrap) folded into the gathered
// vector.  Used by the one-system FP64 kernels: 36 doubles of links in
// registers instead of 72, twice the resident warps for an FP64-bound
// kernel.
template <int PREC, int RECON, int NR, int MODE>
__device__ __forceinline__ void pair_hops(const DslashArgs &a, const LinkScales &ls,
                                          const SiteCoords &sc, int i, int r0,
                                          const bool (&active)[NR],
                                          Vec3<typename AccumType<PREC>::R> (&acc)[NR]) {
  using R = typename AccumType<PREC>::R;
  const Geom &g = a.g;
  const int S = g.stride;
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    int nb[4];
    float f[4];
    nb[0] = hop<+1>(g, sc, mu, f[0]);
    nb[1] = hop<-1>(g, sc, mu, f[1]);
    nb[2] = hop<+3>(g, sc, mu, f[2]);
    nb[3] = hop<-3>(g, sc, mu, f[3]);
    const float eta = eta_sign(sc, mu);
    f[0] *= eta;
    f[1] *= -eta;
    f[2] *= eta;
    f[3] *= -eta;
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      Mat3<R> m[2];
      if (kind == 0) LinkIO<PREC, RECON>::template load_pair<0>(a.links, S, i, mu, ls, m);
      else LinkIO<PREC, RECON>::template load_pair<1>(a.links, S, i, mu, ls, m);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (!active[r]) continue;
        const char *in = a.in + (size_t)(r0 + r) * a.in_fb;
        const char *fx = (a.xs != nullptr) ? a.xs + (size_t)(r0 + r) * a.xs_fb : nullptr;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const Vec3<R> v =
              gather_in<PREC, MODE, R>(in, fx, a.xs_prec, S, nb[2 * kind + h], f[2 * kind + h]);
          mat_vec_acc(acc[r], m[h], v);
        }
      }
    }
  }
}

// ------------------------------------------------ many systems per thread
// FP32 tiles of NR >= 2 systems.  The link stream is staged in shared
// memory: every thread copies its own site's planes there with cp.async (16
// bytes per plane, L2 evict-first) and reads only what it copied itself, so
// no thread waits for another -- only for its own copy groups
// (cp.async.wait_group).  The stage holds one direction, as two halves: the
// fat pair (planes 0-8) and the long pair (planes 9 on); each half of
// direction mu + 1 is copied while the other half of direction mu is
// multiplied.  The registers left free hold NR systems' accumulators.  One
// hop matrix is read at a time (18 floats), the hop's sign (eta, backward
// hop, antiperiodic wrap) is folded into it once, and it is applied to the
// gathered neighbour vector of every system of the tile, so the per-system
// work is the 16 gathers and the 16 x 18 packed FFMA2 of the mat-vecs.
// Shared memory: NPL planes x 16 bytes per thread (NPL = 18 for 18-real long
// links, 15 for 12-real).  A stage of two directions measured 10-12 % slower
// at 24^3 x 64 with 12 systems: its 221 KB per SM left L1 28 KB for the
// gathered neighbours.
template <int RECON> struct StagedPlanes {
  static constexpr int n = LinkLayout<PREC_F32, RECON>::mu_bytes / 16;
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;"
               :: "r"(s), "l"(gsrc), "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

// Copy half HALF (0: the fat pair's planes 0-8, 1: the long pair's planes 9
// to NPL - 1) of direction mu at site i into the stage `buf` (this thread's
// column of it) and commit it as one group.
template <int RECON, int HALF>
__device__ __forceinline__ void stage_half(const char *links, int S, int i, int mu, float4 *buf,
                                           uint64_t pol) {
  constexpr int NPL = StagedPlanes<RECON>::n;
  constexpr int p0 = HALF ? 9 : 0, p1 = HALF ? NPL : 9;
  const char *src = links + ((size_t)mu * NPL * S + i) * 16;
#pragma unroll
  for (int p = p0; p < p1; ++p)
    cp_async16(buf + p * blockDim.x + threadIdx.x, src + (size_t)p * S * 16, pol);
  cp_async_commit();
}

// Hop matrix H (0: F(x), 1: F(x-mu)^dag, 2: L(x), 3: L(x-3mu)^dag) of the
// staged direction `buf`.  The two matrices of a pair share its middle plane.
template <int RECON, int H>
__device__ __forceinline__ void staged_hop(const float4 *buf, const LinkScales &ls,
                                           Mat3<float> &m) {
  constexpr bool k12 = (H >= 2 && RECON == 12);
  constexpr int ne = k12 ? 6 : 9;
  constexpr int base = (H >= 2) ? 9 : 0;  // first plane of the pair
  const int T = blockDim.x;
  const float4 *b = buf + threadIdx.x;
  float f[20];
  if constexpr (k12) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 q = b[(base + 3 * (H - 2) + k) * T];
      f[4 * k] = q.x; f[4 * k + 1] = q.y; f[4 * k + 2] = q.z; f[4 * k + 3] = q.w;
    }
  } else if constexpr ((H & 1) == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const float4 q = b[(base + k) * T];
      f[4 * k] = q.x; f[4 * k + 1] = q.y; f[4 * k + 2] = q.z; f[4 * k + 3] = q.w;
    }
  } else {
    {
      const float4 q = b[(base + 4) * T];
      f[0] = q.z; f[1] = q.w;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 q = b[(base + 5 + k) * T];
      f[2 + 4 * k] = q.x; f[3 + 4 * k] = q.y; f[4 + 4 * k] = q.z; f[5 + 4 * k] = q.w;
    }
  }
#pragma unroll
  for (int e = 0; e < ne; ++e) m.e[e] = make_float2(f[2 * e], f[2 * e + 1]);
  if constexpr (k12) reconstruct_row2(m, ls.recon_f);
}

// Neighbour colour vectors of NR systems at the two hops of one pair (the
// hops' sites nb0, nb1), into registers; inactive systems are skipped.
template <int NR>
__device__ __forceinline__ void gather_pair(const DslashArgs &a, int S, int r0,
                                            const bool (&active)[NR], int nb0, int nb1,
                                            Vec3<float> (&v)[2][NR]) {
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (!active[r]) continue;
    const char *f = a.in + (size_t)(r0 + r) * a.in_fb;
    v[0][r] = SpinorIO<PREC_F32>::load(f, S, nb0);
    v[1][r] = SpinorIO<PREC_F32>::load(f, S, nb1);
  }
}

// acc_r += (s0 M0) v[0][r] + (s1 M1) v[1][r] for one staged pair, in packed
// FP32 pairs: with A = s M_ij = (a, b) and A' = (-b, a),
//   (M v)_i += A (Re v_j, Re v_j) + A' (Im v_j, Im v_j),
// two FFMA2 per complex multiply-add with one real part of the vector in both
// lanes, half the FMA instructions of the scalar form.  A and A' are formed
// once per tile (FMUL2) and serve every system of it.
template <int RECON, int KIND, int NR>
__device__ __forceinline__ void apply_pair(const float4 *buf, const LinkScales &ls, float s0,
                                           float s1, const bool (&active)[NR],
                                           const Vec3<float> (&v)[2][NR],
                                           Vec3<float> (&acc)[NR]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    Mat3<float> m;
    if (h == 0) staged_hop<RECON, 2 * KIND>(buf, ls, m);
    else staged_hop<RECON, 2 * KIND + 1>(buf, ls, m);
    const float sg = h ? s1 : s0;
    // row by row: the two forms of one row (12 registers) are live at a time
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float2 A[3], B[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 e = m.e[3 * i + j];
        A[j] = __fmul2_rn(e, make_float2(sg, sg));
        B[j] = __fmul2_rn(make_float2(e.y, e.x), make_float2(-sg, sg));
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (!active[r]) continue;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float2 vj = v[h][r].c[j];
          acc[r].c[i] = __ffma2_rn(A[j], make_float2(vj.x, vj.x), acc[r].c[i]);
          acc[r].c[i] = __ffma2_rn(B[j], make_float2(vj.y, vj.y), acc[r].c[i]);
        }
      }
    }
  }
}

// Own-site vectors of the epilogue, staged in the fat half of the stage once
// direction 3's fat pair is multiplied, so their load latency hides behind
// its long pair.  Vector v (in the order p, xs, r of the tile's systems;
// NORM stages the input at the own index as p) keeps its 16-byte part in
// slot v and its 8-byte part in half (v & 1) of slot V + v / 2; as many as
// fit the half (9 slots per thread) are staged, the rest go to registers
// (EpiRest).
template <int MODE, int NR> struct EpiVecs {
  static constexpr int nvec = (MODE == MODE_UPDATE) ? 3 : (MODE == MODE_NORM || MODE == MODE_MDAGM) ? 1 : 0;
  static constexpr int total = nvec * NR;
};
template <int MODE, int RECON, int NR> struct EpiStage {
  static constexpr int cap = 2 * 9 / 3;
  static constexpr int V = EpiVecs<MODE, NR>::total < cap ? EpiVecs<MODE, NR>::total : cap;
};

__device__ __forceinline__ void cp_async16_vec(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(s), "l"(gsrc) : "memory");
}

// Field of epilogue vector v: the base of system r0 + v % NR's colour vector.
template <int MODE, int NR>
__device__ __forceinline__ const char *epi_field(const DslashArgs &a, int r0, int v) {
  const int k = v / NR, r = r0 + v % NR;
  if constexpr (MODE == MODE_NORM) return a.in + (size_t)r * a.in_fb;
  if (k == 0) return a.p + (size_t)r * a.p_fb;
  if (k == 1) return a.xs + (size_t)r * a.xs_fb;
  return a.out + (size_t)r * a.out_fb;
}

template <int MODE, int RECON, int NR>
__device__ __forceinline__ void stage_epilogue(const DslashArgs &a, int S, int i, int r0,
                                               const bool (&active)[NR], float4 *buf) {
  constexpr int V = EpiStage<MODE, RECON, NR>::V;
  if constexpr (V > 0) {
    const int T = blockDim.x, t = threadIdx.x;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (!active[v % NR]) continue;
      const char *f = epi_field<MODE, NR>(a, r0, v);
      cp_async16_vec(buf + v * T + t, f + (size_t)i * 16);
      cp_async8(reinterpret_cast<char *>(buf + (V + v / 2) * T + t) + 8 * (v & 1),
                f + (size_t)16 * S + (size_t)i * 8);
    }
    cp_async_commit();
  }
}

// The caller staged both halves of direction 0 (two commit groups) before
// waiting for its predecessor kernel.  One pair's gathers (2 hops x NR
// systems) are in flight while the previous pair is multiplied: the loop is
// bound by the latency of the L2 gathers, and this keeps about twice as many
// in flight per thread as gathering hop by hop.  (Tiles of 6, 8 and 12
// systems, which gathered hop by hop for want of registers, measured 1.7x
// slower than 4 at 24^3 x 64 with 12 systems.)
// The epilogue's own-site vectors that do not fit the stage (mode 4: 6 of
// its 12) are loaded during direction 3's long pair into the fat-pair gather
// buffer, which has no next direction to hold: vector V + k in slot
// [k / NR][k % NR].
template <int MODE, int RECON, int NR> struct EpiRest {
  static constexpr int n = EpiVecs<MODE, NR>::total - EpiStage<MODE, RECON, NR>::V;
  static_assert(n <= 2 * NR, "the rest of the epilogue vectors fits the fat-pair buffer");
  __device__ __forceinline__ static void load(const DslashArgs &a, int S, int i, int r0,
                                              const bool (&active)[NR], Vec3<float> (&buf)[2][NR]) {
    constexpr int V = EpiStage<MODE, RECON, NR>::V;
#pragma unroll
    for (int k = 0; k < n; ++k)
      if (active[(V + k) % NR])
        buf[k / NR][k % NR] = SpinorIO<PREC_F32>::load(epi_field<MODE, NR>(a, r0, V + k), S, i);
  }
};

// Epilogue vector v of this thread: from the stage, or from the fat-pair
// buffer the last direction loaded it into.
template <int MODE, int RECON, int NR>
__device__ __forceinline__ Vec3<float> epi_vec(const float4 *stage, const Vec3<float> (&buf)[2][NR],
                                               int v) {
  constexpr int V = EpiStage<MODE, RECON, NR>::V;
  if (v < V) {
    const int T = blockDim.x, t = threadIdx.x;
    const float4 q = stage[v * T + t];
    const float2 w = reinterpret_cast<const float2 *>(stage + (V + v / 2) * T + t)[v & 1];
    Vec3<float> o;
    o.c[0] = make_float2(q.x, q.y);
    o.c[1] = make_float2(q.z, q.w);
    o.c[2] = w;
    return o;
  }
  return buf[(v - V) / NR][(v - V) % NR];
}

// The caller staged both halves of direction 0 (two commit groups) before
// waiting for its predecessor kernel.  One pair's gathers (2 hops x NR
// systems) are in flight while the previous pair is multiplied: the loop is
// bound by the latency of the L2 gathers, and this keeps about twice as many
// in flight per thread as gathering hop by hop.  (Tiles of 6, 8 and 12
// systems, which gathered hop by hop for want of registers, measured 1.7x
// slower than 4 at 24^3 x 64 with 12 systems.)  vf, the fat-pair buffer,
// holds the epilogue's unstaged own-site vectors on return; with EARLY it
// arrives with direction 0's fat-pair gathers already issued.
template <int RECON, int NR, int MODE, bool EARLY>
__device__ __forceinline__ void multi_hops(const DslashArgs &a, const LinkScales &ls,
                                           const SiteCoords &sc, int i, int r0,
                                           const bool (&active)[NR], Vec3<float> (&acc)[NR],
                                           float4 *stage, Vec3<float> (&vf)[2][NR]) {
  const Geom &g = a.g;
  const int S = g.stride;
  const uint64_t pol = l2_link_policy(ls.keep);
  static_assert(NR <= 4, "FP32 tiles hold 1, 2 or 4 systems");
  constexpr bool kEpi = EpiStage<MODE, RECON, NR>::V > 0;
  Vec3<float> vl[2][NR];  // long pair
  if constexpr (!EARLY) {  // else the caller has issued them
    float d0, d1;
    gather_pair<NR>(a, S, r0, active, hop<+1>(g, sc, 0, d0), hop<-1>(g, sc, 0, d1), vf);
  }
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    float f[4];
    const int n2 = hop<+3>(g, sc, mu, f[2]);
    const int n3 = hop<-3>(g, sc, mu, f[3]);
    hop<+1>(g, sc, mu, f[0]);
    hop<-1>(g, sc, mu, f[1]);
    const float eta = eta_sign(sc, mu);
    gather_pair<NR>(a, S, r0, active, n2, n3, vl);
    // copy groups in flight: [fat mu, long mu]; wait for the fat half
    cp_async_wait<1>();
    apply_pair<RECON, 0, NR>(stage, ls, eta * f[0], -eta * f[1], active, vf, acc);
    // the fat half is read: it takes direction mu + 1's fat pair, or after
    // direction 3 the epilogue's own-site vectors
    if (mu < 3) {
      stage_half<RECON, 0>(a.links, S, i, mu + 1, stage, pol);
      float d0, d1;
      gather_pair<NR>(a, S, r0, active, hop<+1>(g, sc, mu + 1, d0),
                      hop<-1>(g, sc, mu + 1, d1), vf);
    } else {
      stage_epilogue<MODE, RECON, NR>(a, S, i, r0, active, stage);
      EpiRest<MODE, RECON, NR>::load(a, S, i, r0, active, vf);
    }
    // in flight: [long mu, next group]; wait for the long half
    if (mu < 3 || kEpi) cp_async_wait<1>();
    else cp_async_wait<0>();
    apply_pair<RECON, 1, NR>(stage, ls, eta * f[2], -eta * f[3], active, vl, acc);
    if (mu < 3) stage_half<RECON, 1>(a.links, S, i, mu + 1, stage, pol);
  }
}

// Direction 0's links of a site, loaded before the kernel waits for its
// predecessor (links never change during a solve).  FP64 kernels do not
// prefetch: the reliable-update pair is idle in most checkpoints, and would
// stream a quarter of its links for nothing.
template <int PREC, int RECON> struct FirstLinks {
  static constexpr bool kUsed = (PREC == PREC_F32);
  Mat3<typename AccumType<PREC>::R> m[4];
  __device__ __forceinline__ void load(const DslashArgs &a, const LinkScales &ls, int i) {
    LinkIO<PREC, RECON>::load(a.links, a.g.stride, i, 0, ls, m);
  }
};
template <int RECON> struct FirstLinks<PREC_I16, RECON> {
  static constexpr bool kUsed = true;
  I16Words<RECON> buf;
  __device__ __forceinline__ void load(const DslashArgs &a, const LinkScales &ls, int i) {
    i16_load_words<RECON>(a.links, a.g.stride, i, 0, buf, ls.keep);
  }
};

// Launch bounds per precision: FP64 needs the large register file of the SM
// (a 512-thread bound squeezes it to 64 registers and spills); FP32 and
// 16-bit fit 128 registers at up to 512 threads.
template <int PREC, int NR> struct DslashBounds {
  static constexpr int threads = (PREC == PREC_F64) ? 256 : 512;
  static constexpr int min_blocks = 1;
};
// FP32 tiles of several systems: three 128-thread blocks per SM (up to 168
// registers; the staged links take 288 bytes of shared memory per thread)
template <int NR> struct DslashBounds<PREC_F32, NR> {
  static constexpr int threads = (NR == 1) ? 512 : 128;
  static constexpr int min_blocks = (NR == 1) ? 1 : 3;
};
// One-RHS 16-bit: six 128-thread blocks per SM (at most 85 registers): the
// kernel is latency-bound and gains more from resident warps than from
// registers.
template <> struct DslashBounds<PREC_I16, 1> {
  static constexpr int threads = 128, min_blocks = 6;
};
// One-RHS FP64: four 128-thread blocks per SM (at most 128 registers) for
// the pair-at-a-time path.
template <> struct DslashBounds<PREC_F64, 1> {
  static constexpr int threads = 128, min_blocks = 4;
};
// Largest block a (precision, RHS tile) kernel may be launched with.
inline int dslash_max_block(int prec, int nr) {
  if (prec == PREC_I16 && nr == 1) return DslashBounds<PREC_I16, 1>::threads;
  if (prec == PREC_F64 && nr == 1) return DslashBounds<PREC_F64, 1>::threads;
  if (prec == PREC_F32) return nr == 1 ? DslashBounds<PREC_F32, 1>::threads
                                       : DslashBounds<PREC_F32, 2>::threads;
  return prec == PREC_F64 ? DslashBounds<PREC_F64, 2>::threads : DslashBounds<PREC_I16, 2>::threads;
}
// Dynamic shared memory of a launch: the staged links of the FP32 tiles of
// several systems (one direction's planes x 16 bytes per thread).
inline size_t dslash_smem_bytes(int prec, int recon, int nr, int block) {
  if (prec != PREC_F32 || nr == 1) return 0;
  const int npl = (recon == 12) ? 15 : 18;
  return (size_t)npl * 16 * block;
}

// One work item of the kernel: RHS tile blk % ntiles of the blockDim.x
// sites from (blk / ntiles) * blockDim.x on.  A return ends the item.
template <int PREC, int RECON, int NR, int MODE, int OUTP>
__device__ __forceinline__ void dslash_item(const DslashArgs &a, const unsigned blk) {
  using R = typename AccumType<PREC>::R;
  const Geom &g = a.g;
  const int S = g.stride;
  // Blocks of the RHS tiles of one range of sites are adjacent in the launch
  // order, so the tiles after the first find that range's links in L2.
  const int ntiles = (a.nrhs + NR - 1) / NR;
  const int tile = blk % ntiles;
  const int i = (blk / ntiles) * blockDim.x + threadIdx.x;
  const int r0 = tile * NR;
  LinkScales ls = a.ls;
  ls.keep = tile < ntiles - 1;  // a later tile of this site range reads the links again

  // Work that needs nothing from the predecessor kernel runs before waiting
  // for it: direction 0's links (one-RHS and small tiles) and, for the m^2
  // epilogue, the own-site p, which the kernel two launches back wrote (every
  // kernel lets its successor launch only after its own wait, so that one
  // has completed).
  FirstLinks<PREC, RECON> first;
  constexpr bool kFirst = FirstLinks<PREC, RECON>::kUsed && (PREC == PREC_I16 || NR == 1);
  if constexpr (kFirst) {
    if (i < g.vh) first.load(a, ls, i);
  }
  // FP32 tiles of several systems stage direction 0 of their links in
  // shared memory (see multi_hops)
  constexpr bool kStaged = (PREC == PREC_F32 && NR >= 2);
  extern __shared__ float4 dyn_smem[];
  if constexpr (kStaged) {
    if (i < g.vh) {
      const uint64_t pol = l2_link_policy(ls.keep);
      stage_half<RECON, 0>(a.links, S, i, 0, dyn_smem, pol);
      stage_half<RECON, 1>(a.links, S, i, 0, dyn_smem, pol);
    }
  }

  constexpr bool kPreP = (MODE == MODE_MDAGM || MODE == MODE_UPDATE) && NR < 8 && !kStaged;
  Vec3<R> pre[kPreP ? NR : 1];
  if constexpr (kPreP) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (i < g.vh && r0 + r < a.nrhs)
        pre[r] = SpinorIO<PREC>::load(a.p + (size_t)(r0 + r) * a.p_fb, S, i);
      else
        zero(pre[r]);
    }
  }
  // UPDATE: r and xs were last written three or more kernels back as well
  // (prefetched where registers allow)
  constexpr int XP = (PREC == PREC_F64) ? PREC_F64 : PREC_F32;
  using RX = typename SpinorIO<XP>::R;
  constexpr bool kPreRX = (MODE == MODE_UPDATE) && NR == 1 && PREC != PREC_F64;  // registers
  Vec3<R> pre_r[kPreRX ? NR : 1];
  Vec3<RX> pre_x[kPreRX ? NR : 1];
  if constexpr (kPreRX) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (i < g.vh && r0 + r < a.nrhs) {
        pre_r[r] = SpinorIO<PREC>::load(a.out + (size_t)(r0 + r) * a.out_fb, S, i);
        pre_x[r] = SpinorIO<XP>::load(a.xs + (size_t)(r0 + r) * a.xs_fb, S, i);
      } else {
        zero(pre_r[r]);
        zero(pre_x[r]);
      }
    }
  }
  griddep_wait();
  griddep_launch_dependents();

  // Staged tiles: direction 0's fat-pair gathers (every system of the tile)
  // go out before the gate is read, so that their latency overlaps the
  // gate's -- for the update kernel only: D_eo 311 -> 302-309 us with 12
  // systems at 24^3 x 64, while the plain and D_oe kernels lost 12-27 us
  // with it.  (A tile the gate then skips has loaded for nothing.)
  constexpr bool kEarly = kStaged && MODE == MODE_UPDATE;
  Vec3<float> vbuf[kStaged ? 2 : 1][kStaged ? NR : 1];  // staged tiles: the fat-pair gathers
  if constexpr (kEarly) {
    if (i < g.vh) {
      const SiteCoords sc = site_coords(g, a.out_parity, i);
      bool all[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) all[r] = r0 + r < a.nrhs;
      float d0, d1;
      gather_pair<NR>(a, S, r0, all, hop<+1>(g, sc, 0, d0), hop<-1>(g, sc, 0, d1), vbuf);
    }
  }

  // Gate: the decision is the same in every block of a tile row (a system's
  // state only changes in a later kernel -- a finish kernel -- or in the
  // warp that completes an in-kernel reduction over its row, after every
  // block of the row has read it).  Rows are independent.
  bool active[NR];
  bool any_here = false;
  if (a.slots != nullptr && a.gate != GATE_NONE) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      active[r] = (r0 + r < a.nrhs) && slot_active(a.slots + r0 + r, a.gate);
      any_here |= active[r];
    }
    if (!any_here) {
      if constexpr (kStaged) cp_async_wait<0>();  // no copy outlives its thread
      return;
    }
  } else {
#pragma unroll
    for (int r = 0; r < NR; ++r) active[r] = (r0 + r < a.nrhs);
    any_here = true;
  }
  const bool valid = (i < g.vh) && any_here;

  Vec3<R> acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) zero(acc[r]);

  if (valid) {
    const SiteCoords sc = site_coords(g, a.out_parity, i);
    if constexpr (PREC == PREC_I16) {
      i16_hops<RECON, NR>(a, ls, sc, i, r0, active, acc, first.buf);
    } else if constexpr (kStaged) {
      multi_hops<RECON, NR, MODE, kEarly>(a, ls, sc, i, r0, active, acc, dyn_smem, vbuf);
      if constexpr (EpiStage<MODE, RECON, NR>::V > 0) cp_async_wait<0>();
    } else if constexpr (PREC == PREC_F64 && NR == 1) {
      pair_hops<PREC, RECON, NR, MODE>(a, ls, sc, i, r0, active, acc);
    } else {
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
        Mat3<R>(&m)[4] = first.m;  // direction 0 arrived before the wait
        if (!kFirst || mu > 0) LinkIO<PREC, RECON>::load(a.links, S, i, mu, ls, m);
        float sg[4];
        int nb[4];
        nb[0] = hop_index(g, sc, mu, +1, sg[0]);
        nb[1] = hop_index(g, sc, mu, -1, sg[1]);
        nb[2] = hop_index(g, sc, mu, +3, sg[2]);
        nb[3] = hop_index(g, sc, mu, -3, sg[3]);
        const float eta = eta_sign(sc, mu);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (!active[r]) continue;
          const char *f = a.in + (size_t)(r0 + r) * a.in_fb;
          const char *fx = (a.xs != nullptr) ? a.xs + (size_t)(r0 + r) * a.xs_fb : nullptr;
          Vec3<R> t;
          zero(t);
          Vec3<R> v;
          v = gather_in<PREC, MODE, R>(f, fx, a.xs_prec, S, nb[0], sg[0]);
          mat_vec_acc(t, m[0], v);
          v = gather_in<PREC, MODE, R>(f, fx, a.xs_prec, S, nb[1], sg[1]);
          mat_vec_sub(t, m[1], v);
          v = gather_in<PREC, MODE, R>(f, fx, a.xs_prec, S, nb[2], sg[2]);
          mat_vec_acc(t, m[2], v);
          v = gather_in<PREC, MODE, R>(f, fx, a.xs_prec, S, nb[3], sg[3]);
          mat_vec_sub(t, m[3], v);
          if (eta > 0.f) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { acc[r].c[c].x += t.c[c].x; acc[r].c[c].y += t.c[c].y; }
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) { acc[r].c[c].x -= t.c[c].x; acc[r].c[c].y -= t.c[c].y; }
          }
        }
      }
    }
  }

  if constexpr (MODE == MODE_PLAIN) {
    if (valid) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (!active[r]) continue;
        Vec3<R> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) { o.c[c].x = R(0.5) * acc[r].c[c].x; o.c[c].y = R(0.5) * acc[r].c[c].y; }
        SpinorIO<PREC>::store(a.out + (size_t)(r0 + r) * a.out_fb, S, i, o);
      }
    }
  } else if constexpr (MODE == MODE_MDAGM) {
    // Ap = m^2 p - 1/2 acc ; partial Re<p, Ap>
    R dot[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      dot[r] = 0;
      if (valid && active[r]) {
        const R m2 = (R)(a.slots ? a.slots[r0 + r].m2 : a.m2_const);
        Vec3<R> p;
        if constexpr (kPreP) p = pre[r];
        else if constexpr (kStaged) p = epi_vec<MODE, RECON, NR>(dyn_smem, vbuf, r);
        else p = SpinorIO<PREC>::load(a.p + (size_t)(r0 + r) * a.p_fb, S, i);
        Vec3<R> o;
        R d = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          o.c[c].x = fma(m2, p.c[c].x, R(-0.5) * acc[r].c[c].x);
          o.c[c].y = fma(m2, p.c[c].y, R(-0.5) * acc[r].c[c].y);
          d = fma(p.c[c].x, o.c[c].x, d);
          d = fma(p.c[c].y, o.c[c].y, d);
        }
        SpinorIO<PREC>::store(a.out + (size_t)(r0 + r) * a.out_fb, S, i, o);
        dot[r] = d;
      }
    }
    if (a.slots != nullptr && a.partial != nullptr && any_here) {
      // <p, Ap> of every system of this tile; the warp completing the sums
      // sets alpha for the tile's running systems
      double *inst[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r)
        inst[r] = a.partial + (size_t)min(r0 + r, a.nrhs - 1) * red_stride(g);
      double pap[NR];
      if (warp_tree_reduce<NR>(dot, min(NR, a.nrhs - r0), inst, g, i,
                               a.counter + (size_t)tile * ticket_stride(g), pap) &&
          (threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (!active[r]) continue;
          finish_alpha(a.slots + r0 + r, pap[r]);
          if (a.shifts) finish_shift_alpha(a.slots + r0 + r, a.shifts, a.nshift);
        }
      }
    }
  } else if constexpr (MODE == MODE_NORM) {
    // t = D p ; partial |t|^2 + m^2 |p|^2 (p at the own index of the input
    // parity: every input site is counted once)
    R val[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      val[r] = 0;
      if (valid && active[r]) {
        Vec3<R> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) { o.c[c].x = R(0.5) * acc[r].c[c].x; o.c[c].y = R(0.5) * acc[r].c[c].y; }
        SpinorIO<PREC>::store(a.out + (size_t)(r0 + r) * a.out_fb, S, i, o);
        Vec3<R> p;
        if constexpr (kStaged) p = epi_vec<MODE, RECON, NR>(dyn_smem, vbuf, r);
        else p = SpinorIO<PREC>::load(a.in + (size_t)(r0 + r) * a.in_fb, S, i);
        R no = 0, np = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          no = fma(o.c[c].x, o.c[c].x, fma(o.c[c].y, o.c[c].y, no));
          np = fma(p.c[c].x, p.c[c].x, fma(p.c[c].y, p.c[c].y, np));
        }
        val[r] = fma((R)a.slots[r0 + r].m2, np, no);
      }
    }
    if (a.slots != nullptr && a.partial != nullptr && any_here) {
      double *inst[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r)
        inst[r] = a.partial + (size_t)min(r0 + r, a.nrhs - 1) * red_stride(g);
      warp_partials<NR>(val, min(NR, a.nrhs - r0), inst, g, i);
    }
  } else if constexpr (MODE == MODE_UPDATE) {
    // Ap = m^2 p - 1/2 acc ; xs += alpha p ; r -= alpha Ap ; partial |r|^2
    R val[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      val[r] = 0;
      if (valid && active[r]) {
        const SlotState *sl = a.slots + r0 + r;
        const R m2 = (R)sl->m2, al = (R)sl->alpha;
        Vec3<R> p, rv;
        Vec3<RX> xv;
        if constexpr (kPreP) p = pre[r];
        else if constexpr (kStaged) p = epi_vec<MODE, RECON, NR>(dyn_smem, vbuf, r);
        else p = SpinorIO<PREC>::load(a.p + (size_t)(r0 + r) * a.p_fb, S, i);
        if constexpr (kPreRX) {
          rv = pre_r[r];
          xv = pre_x[r];
        } else if constexpr (kStaged) {
          xv = epi_vec<MODE, RECON, NR>(dyn_smem, vbuf, NR + r);
          rv = epi_vec<MODE, RECON, NR>(dyn_smem, vbuf, 2 * NR + r);
        } else {
          rv = SpinorIO<PREC>::load(a.out + (size_t)(r0 + r) * a.out_fb, S, i);
          xv = SpinorIO<XP>::load(a.xs + (size_t)(r0 + r) * a.xs_fb, S, i);
        }
        R n2 = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const R apx = fma(m2, p.c[c].x, R(-0.5) * acc[r].c[c].x);
          const R apy = fma(m2, p.c[c].y, R(-0.5) * acc[r].c[c].y);
          xv.c[c].x = fma((RX)al, (RX)p.c[c].x, xv.c[c].x);
          xv.c[c].y = fma((RX)al, (RX)p.c[c].y, xv.c[c].y);
          rv.c[c].x = fma(-al, apx, rv.c[c].x);
          rv.c[c].y = fma(-al, apy, rv.c[c].y);
          n2 = fma(rv.c[c].x, rv.c[c].x, fma(rv.c[c].y, rv.c[c].y, n2));
        }
        SpinorIO<XP>::store(a.xs + (size_t)(r0 + r) * a.xs_fb, S, i, xv);
        SpinorIO<PREC>::store(a.out + (size_t)(r0 + r) * a.out_fb, S, i, rv);
        val[r] = n2;
      }
    }
    if (a.slots != nullptr && a.partial != nullptr && any_here) {
      double *inst[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r)
        inst[r] = a.partial + (size_t)min(r0 + r, a.nrhs - 1) * red_stride(g);
      warp_partials<NR>(val, min(NR, a.nrhs - r0), inst, g, i);
    }

  } else {  // MODE_RESID (PREC == F64)
    double val[3][NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      val[0][r] = val[1][r] = val[2][r] = 0.0;
      if (valid && active[r]) {
        const double m2 = a.slots[r0 + r].m2;
        Vec3<double> x = SpinorIO<PREC_F64>::load(a.x64 + (size_t)(r0 + r) * a.f64_fb, S, i);
        if (a.xs != nullptr) {  // fold the sloppy increment: x64 += xs, xs = 0
          char *fx = a.xs + (size_t)(r0 + r) * a.xs_fb;
          if (a.xs_prec == PREC_F32) {
            Vec3<float> d = SpinorIO<PREC_F32>::load(fx, S, i), z;
#pragma unroll
            for (int c = 0; c < 3; ++c) { x.c[c].x += (double)d.c[c].x; x.c[c].y += (double)d.c[c].y; }
            zero(z);
            SpinorIO<PREC_F32>::store(fx, S, i, z);
          } else {
            Vec3<double> d = SpinorIO<PREC_F64>::load(fx, S, i), z;
#pragma unroll
            for (int c = 0; c < 3; ++c) { x.c[c].x += d.c[c].x; x.c[c].y += d.c[c].y; }
            zero(z);
            SpinorIO<PREC_F64>::store(fx, S, i, z);
          }
          SpinorIO<PREC_F64>::store(const_cast<char *>(a.x64) + (size_t)(r0 + r) * a.f64_fb, S, i, x);
        }
        Vec3<double> b = SpinorIO<PREC_F64>::load(a.b64 + (size_t)(r0 + r) * a.f64_fb, S, i);
        Vec3<double> rr;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rr.c[c].x = b.c[c].x - fma(m2, x.c[c].x, -0.5 * (double)acc[r].c[c].x);
          rr.c[c].y = b.c[c].y - fma(m2, x.c[c].y, -0.5 * (double)acc[r].c[c].y);
        }
        using RO = typename SpinorIO<OUTP>::R;
        Vec3<RO> p = SpinorIO<OUTP>::load(a.ps + (size_t)(r0 + r) * a.ps_fb, S, i);
        double n2 = 0, pre = 0, pim = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          n2 = fma(rr.c[c].x, rr.c[c].x, fma(rr.c[c].y, rr.c[c].y, n2));
          // <r, p> = sum conj(r) p
          pre = fma(rr.c[c].x, (double)p.c[c].x, fma(rr.c[c].y, (double)p.c[c].y, pre));
          pim = fma(rr.c[c].x, (double)p.c[c].y, fma(-rr.c[c].y, (double)p.c[c].x, pim));
        }
        SpinorIO<OUTP>::store(a.out + (size_t)(r0 + r) * a.out_fb, S, i, convert<RO>(rr));
        val[0][r] = n2; val[1][r] = pre; val[2][r] = pim;
      }
    }
    if (any_here) {
      // |r|^2, <r, p> of every system of this tile (value k*3 + v); the warp
      // completing the sums finishes the tile's reliable updates
      double vals[3 * NR];
      double *inst[3 * NR];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          vals[3 * r + v] = val[v][r];
          inst[3 * r + v] =
              a.partial + ((size_t)v * a.nrhs + min(r0 + r, a.nrhs - 1)) * red_stride(g);
        }
      double out[3 * NR];
      if (warp_tree_reduce<3 * NR>(vals, 3 * min(NR, a.nrhs - r0), inst, g, i,
                                   a.counter + (size_t)tile * ticket_stride(g), out) &&
          (threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (active[r])
            finish_reliable_update(a.slots + r0 + r, out[3 * r], out[3 * r + 1], out[3 * r + 2]);
      }
    }
  }
}

// Work items of a launch: site blocks x RHS tiles.
__host__ __device__ inline int dslash_items(const Geom &g, int nrhs, int nr, int block) {
  return ((g.vh + block - 1) / block) * ((nrhs + nr - 1) / nr);
}

// Tiles (of NR systems, at most 64) with a system the gate lets through.
template <int NR>
__device__ __forceinline__ unsigned long long active_tiles(const DslashArgs &a, int ntiles) {
  unsigned long long m = 0;
  for (int t = 0; t < ntiles; ++t) {
    bool any = a.slots == nullptr || a.gate == GATE_NONE;
    for (int r = t * NR; r < min(a.nrhs, (t + 1) * NR) && !any; ++r)
      any = slot_active(a.slots + r, a.gate);
    if (any) m |= 1ull << t;
  }
  return m;
}

// Position of the j-th (from 0) set bit of m.
__device__ __forceinline__ int nth_bit(unsigned long long m, int j) {
  const unsigned lo = (unsigned)m;
  const int nlo = __popc(lo);
  return j < nlo ? (int)__fns(lo, 0, j + 1) : 32 + (int)__fns((unsigned)(m >> 32), 0, j - nlo + 1);
}

// One block per work item.
template <int PREC, int RECON, int NR, int MODE, int OUTP>
__global__ void __launch_bounds__(DslashBounds<PREC, NR>::threads,
                                  DslashBounds<PREC, NR>::min_blocks)
dslash_kernel(const DslashArgs a) {
  dslash_item<PREC, RECON, NR, MODE, OUTP>(a, blockIdx.x);
}

// Resident blocks per SM of the one-system gated kernels (up to 168
// registers at 128 threads: the loop around the item must not push the FP64
// item into spills).
constexpr int GATED_BLOCKS_PER_SM = 3;

// The FP64 kernels of the reliable-update pair, which have work only at a
// few of their launches, run on a grid of a few blocks per SM
// (DslashArgs::max_grid) that share the items of the tiles the gate lets
// through: item k is site block k / nact of the (k % nact)-th active tile,
// taken by block k % gridDim.x.  An empty launch costs one wave of blocks,
// not a block per item, and when some systems need an update every block
// works on theirs.
template <int RECON, int NR, int MODE, int OUTP>
__global__ void __launch_bounds__(DslashBounds<PREC_F64, NR>::threads,
                                  NR == 1 ? GATED_BLOCKS_PER_SM : DslashBounds<PREC_F64, NR>::min_blocks)
dslash_gated_kernel(const DslashArgs a) {
  griddep_wait();  // the gate reads what the previous kernel wrote
  const int ntiles = (a.nrhs + NR - 1) / NR;
  const unsigned long long act = active_tiles<NR>(a, ntiles);
  const int nact = __popcll(act);
  const int n = nact * ((a.g.vh + (int)blockDim.x - 1) / (int)blockDim.x);
  for (int k = blockIdx.x; k < n; k += gridDim.x)
    dslash_item<PREC_F64, RECON, NR, MODE, OUTP>(a, (k / nact) * ntiles + nth_bit(act, k % nact));
  griddep_launch_dependents();
}

// Host-side launcher (defined per precision in dslash_*.cu).
int launch_dslash(int prec, int recon, int nr, int mode, int outp, const DslashArgs &a,
                  int block, cudaStream_t stream);

}  // namespace sq
