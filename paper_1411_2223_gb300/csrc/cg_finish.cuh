// Scalar steps of the CG recurrences, run by one thread of the last block of
// each reduction kernel so that an iteration needs no host round trip.
//
// CG on A x = b (Hestenes-Stiefel): alpha = rr / <p, A p>, x += alpha p,
// r -= alpha A p, beta = rr_new / rr, p = r + beta p.  The mixed-precision
// variant (the paper's "most of the calculations in single precision", Sec. 2)
// accumulates x in FP64 and recomputes the true residual b - A x in FP64
// when |r| has dropped below delta * max|r| since the last update, when the
// recursion claims convergence, and at max_iter (reliable updates).  After
// such an update the old direction p is made orthogonal to the new residual,
// p <- p - (<r, p> / |r|^2) r, before p = r + beta p.
#pragma once

#include "sq_types.h"

namespace sq {

__device__ __forceinline__ void finish_init(SlotState *s, double b2) {
  s->status = SLOT_RUNNING;
  s->b2 = b2;
  s->tol2b2 = s->tol2 * b2;
  s->rr = b2;
  s->maxr = sqrt(b2);
  s->iter = 0;
  s->n_ru = 0;
  s->alpha = 0;
  s->beta = 0;
  s->a_re = 1;
  s->a_im = 0;
  if (!isfinite(b2)) {
    s->status = SLOT_NONFINITE;
    s->ru_pending = 0;
  } else if (b2 == 0.0) {
    s->status = SLOT_CONVERGED;
    s->rr_true = 0;
    s->ru_pending = 0;
  }
}

__device__ __forceinline__ void finish_alpha(SlotState *s, double pap) {
  if (!isfinite(pap)) {
    s->status = SLOT_NONFINITE;
  } else if (pap > 0.0) {
    s->alpha = s->rr / pap;
  } else {  // p vanished: only a true-residual check can decide
    s->alpha = 0.0;
    s->ru_pending = 1;
  }
}

// Reliable updates run only at checkpoints (every few iterations).  A slot
// whose recursion claims convergence, reaches max_iter or breaks down is
// frozen (SLOT_WAIT) until the next checkpoint decides from the FP64
// residual; a slot whose |r| merely fell below delta * max|r| keeps iterating
// and is updated at the next checkpoint.
__device__ __forceinline__ void finish_update(SlotState *s, double rr_new, int checkpoint) {
  s->iter += 1;
  if (!isfinite(rr_new)) {
    s->status = SLOT_NONFINITE;
    return;
  }
  double rn = sqrt(rr_new);
  if (s->ru_pending || rr_new <= s->tol2b2 || s->iter >= s->max_iter) {
    s->ru_pending = 1;  // beta and rr come from the FP64 residual
    s->status = SLOT_WAIT;
    return;
  }
  if (rn < s->delta * s->maxr) s->ru_want = 1;
  if (checkpoint && s->ru_want) {
    s->ru_pending = 1;
    s->ru_want = 0;
    return;
  }
  s->beta = rr_new / s->rr;
  s->a_re = 1.0;
  s->a_im = 0.0;
  s->rr = rr_new;
  s->maxr = fmax(s->maxr, rn);
}

// rr_true = |b - A x|^2, (rp_re, rp_im) = <r_true, p>
__device__ __forceinline__ void finish_reliable_update(SlotState *s, double rr_true,
                                                       double rp_re, double rp_im) {
  s->ru_pending = 0;
  s->ru_want = 0;
  s->n_ru += 1;
  s->rr_true = rr_true;
  s->status = SLOT_RUNNING;
  if (!isfinite(rr_true)) {
    s->status = SLOT_NONFINITE;
    return;
  }
  if (rr_true <= s->tol2b2) {
    s->status = SLOT_CONVERGED;
    return;
  }
  if (s->iter >= s->max_iter) {
    s->status = SLOT_MAXITER;
    return;
  }
  double beta = (s->rr > 0.0) ? rr_true / s->rr : 0.0;
  s->beta = beta;
  s->a_re = 1.0 - beta * rp_re / rr_true;
  s->a_im = -beta * rp_im / rr_true;
  s->rr = rr_true;
  s->maxr = sqrt(rr_true);
}

// Multi-shift CG (Jegerlehner, hep-lat/9612014): with base coefficients
// alpha_k, beta_k and alpha_{-1} = 1, beta_{-1} = 0, zeta_{-1} = zeta_0 = 1,
//   zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
//                (alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
//                 + zeta_{k-1} alpha_{k-1} (1 + sigma alpha_k)),
//   alpha^s_k = alpha_k zeta_{k+1} / zeta_k,  beta^s_k = beta_k (zeta_{k+1} / zeta_k)^2,
//   x^s += alpha^s_k p^s,  p^s = zeta_{k+1} r_{k+1} + beta^s_k p^s.
// Called after alpha_k of the base system is known.
__device__ __forceinline__ void finish_shift_alpha(SlotState *b, ShiftState *sh, int n) {
  const double al = b->alpha;
  for (int i = 0; i < n; ++i) {
    ShiftState &s = sh[i];
    if (!s.active) continue;
    double den = al * b->beta_prev * (s.zeta_prev - s.zeta) +
                 s.zeta_prev * b->alpha_prev * (1.0 + s.sigma * al);
    s.zeta_next = s.zeta * s.zeta_prev * b->alpha_prev / den;
    s.alpha = al * s.zeta_next / s.zeta;
  }
}

// After |r_{k+1}|^2: beta of every shift, per-shift convergence, rotation of
// the zeta history.  The base keeps iterating while any shift continues.
__device__ __forceinline__ void finish_shift_update(SlotState *b, ShiftState *sh, int n,
                                                    double rr_new) {
  b->iter += 1;
  if (!isfinite(rr_new) || !isfinite(b->alpha)) {
    b->status = SLOT_NONFINITE;
    return;
  }
  const double beta = rr_new / b->rr;
  bool any = false;
  for (int i = 0; i < n; ++i) {
    ShiftState &s = sh[i];
    if (!s.active) continue;
    double ratio = s.zeta_next / s.zeta;
    s.beta = beta * ratio * ratio;
    s.iter = b->iter;
    s.cont = !(s.zeta_next * s.zeta_next * rr_new <= s.tol2b2);
    s.zeta_prev = s.zeta;
    s.zeta = s.zeta_next;
    any |= s.cont != 0;
  }
  b->alpha_prev = b->alpha;
  b->beta_prev = beta;
  b->beta = beta;
  b->rr = rr_new;
  if (!any || b->iter >= b->max_iter) {
    b->final_status = any ? SLOT_MAXITER : SLOT_CONVERGED;
    b->status = SLOT_WAIT;  // the last x updates are still to be applied
  }
}

}  // namespace sq
