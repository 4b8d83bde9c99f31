// Types shared by host and device code of the asqtad CG library.
#pragma once

#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define SQ_HD __host__ __device__
#else
#define SQ_HD
#endif

namespace sq {

enum Prec { PREC_F64 = 0, PREC_F32 = 1, PREC_I16 = 2 };

// Lattice geometry of one gauge field (passed to kernels by value).
struct Geom {
  int L[4];            // Lx, Ly, Lz, Lt (all even)
  int st[4];           // lexicographic strides 1, Lx, Lx*Ly, Lx*Ly*Lz
  int lxh;             // Lx / 2
  int vh;              // sites per parity
  int stride;          // plane stride in sites (vh rounded up to 64)
  int nchunks;         // ceil(vh / CHUNK)
  int nwchunks;        // ceil(vh / 32): one partial per warp of 32 sites
  int ngroups;         // ceil(nwchunks / 32): groups of 32 warp partials
  int t_antiperiodic;  // 1: hops wrapping around t pick up -1
  // exact division by Lx/2, Ly, Lz with a multiply-high (Granlund-Montgomery)
  uint32_t div_m[3];
  int div_s1[3], div_s2[3];
};

// Multiplier and shifts for q = n / d with q = (t + ((n - t) >> s1)) >> s2,
// t = umulhi(n, m): exact for every 32-bit n (Granlund and Montgomery, "Division
// by invariant integers using multiplication", PLDI 1994, Sec. 4).
inline void geom_set_divisor(Geom &g, int k, uint32_t d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  g.div_m[k] = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  g.div_s1[k] = l > 0 ? 1 : 0;
  g.div_s2[k] = l > 0 ? l - 1 : 0;
}

// Doubles of one reduction instance (warp partials, then group sums) and
// unsigned counters of one ticket set (per group, then the final one).
SQ_HD inline size_t red_stride(const Geom &g) { return (size_t)g.nwchunks + g.ngroups; }
SQ_HD inline size_t ticket_stride(const Geom &g) { return (size_t)g.ngroups + 1; }

// Bytes of one packed parity-half colour vector.
inline size_t spinor_bytes(int prec, int stride) {
  return (size_t)stride * (prec == PREC_F64 ? 48 : prec == PREC_F32 ? 24 : 16);
}

// Per right-hand-side CG state, resident on the device.  The reduction
// kernels' last block updates it, so no host round trip sits inside an
// iteration.
enum SlotStatus {
  SLOT_RUNNING = 0,
  SLOT_CONVERGED = 1,
  SLOT_MAXITER = 2,
  SLOT_NONFINITE = 3,
  SLOT_IDLE = 4,  // no system in this slot
  SLOT_WAIT = 5,  // frozen until the next reliable-update checkpoint decides
  SLOT_INIT = 6,  // admitted; the init kernel starts it
};

struct SlotState {
  double m2;        // mass^2 of this system
  double tol2;      // tol^2
  double tol2b2;    // tol^2 |b|^2
  double b2;        // |b|^2
  double rr;        // |r|^2 of the current residual
  double alpha, beta;
  double a_re, a_im;  // p = a r + beta p (a = 1 except after a reliable update)
  double maxr;      // max |r| since the last reliable update
  double rr_true;   // |b - A x|^2 from the last FP64 recomputation
  double delta;     // reliable-update threshold (0: only to confirm convergence)
  int iter;
  int max_iter;
  int n_ru;
  int status;       // SlotStatus
  int ru_pending;   // FP64 true residual to be recomputed at this checkpoint
  int ru_want;      // |r| fell below delta * max|r|: update at the next checkpoint
  // multi-shift CG (base system): previous-iteration coefficients
  double alpha_prev, beta_prev;
  int final_status;  // status taken once the last shifted updates are applied
  int pad;
};

// Per-shift state of multi-shift CG: (A + sigma) x = b shares the Krylov
// space of A; its residual is zeta * r.
struct ShiftState {
  double sigma;                   // m_i^2 - m_base^2 (>= 0)
  double zeta, zeta_prev, zeta_next;
  double alpha, beta;             // shifted CG coefficients of this iteration
  double tol2b2;                  // stop once zeta^2 |r|^2 <= tol^2 |b|^2
  int active;                     // x_i += alpha_i p_i in this iteration
  int cont;                       // p_i continues after this iteration
  int iter;                       // iterations this shift took
  int pad;
};

}  // namespace sq
