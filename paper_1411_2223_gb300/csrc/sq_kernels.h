// Host-side launchers of the library's kernels (all asynchronous).
#pragma once

#include <cuda_runtime.h>

#include "sq_types.h"

namespace sq {

// Arguments of the CG vector kernels (nrhs fields per vector, fb bytes apart).
struct VecArgs {
  Geom g;
  int nrhs;
  char *x64;          // FP64 solution fields
  const char *b64;    // FP64 sources
  size_t f64_fb;
  char *r, *p, *ap;   // sloppy-precision fields
  size_t fb;
  char *xs;           // solution increment since the last reliable update
  size_t xs_fb;       // (FP32, or FP64 for plain FP64 CG)
  SlotState *slots;
  double *partial;
  unsigned *counter;
  int checkpoint;     // finish after the update: a reliable update may follow this iteration
};

// Launch with programmatic stream serialization (the kernel must call
// griddep_wait() before it reads anything the previous kernel wrote).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Precision of the solution increment for a sloppy precision.
inline int xs_prec(int prec) { return prec == PREC_F64 ? PREC_F64 : PREC_F32; }

int launch_cg_xpay(int prec, const VecArgs &a, cudaStream_t st);
int launch_cg_init(int prec, const VecArgs &a, int guess, cudaStream_t st);
// Sum of the per-warp partials the CG's Dslash kernels leave, and the scalar
// step: kind 0 after the D_oe kernel (alpha), 1 after the D_eo kernel (beta,
// convergence, reliable-update request; a.checkpoint).
int launch_cg_finish(int kind, const VecArgs &a, cudaStream_t st);

// canonical complex128 [i][colour] (nrhs fields, canon_elems complex apart)
int launch_pack(int prec, const Geom &g, const double *canon, size_t canon_elems, void *out,
                size_t out_fb, int nrhs, cudaStream_t st);
int launch_unpack(int prec, const Geom &g, const void *in, size_t in_fb, double *canon,
                  size_t canon_elems, int nrhs, cudaStream_t st);
int launch_convert_from_f64(int prec, const Geom &g, const void *in, size_t in_fb, void *out,
                            size_t out_fb, int nrhs, cudaStream_t st);

}  // namespace sq
