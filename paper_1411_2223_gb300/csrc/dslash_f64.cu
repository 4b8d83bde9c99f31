// Instantiations of the Dslash kernel family for PREC_F64 links and vectors.
#include "dslash.cuh"
#include "sq_kernels.h"

namespace sq {

int launch_dslash_f64(int recon, int nr, int mode, int outp, const DslashArgs &a, int block,
                       cudaStream_t st) {
  dim3 grid(dslash_items(a.g, a.nrhs, nr, block));
  // the reliable-update pair: the gated kernel on at most max_grid blocks
  const bool gated = a.max_grid > 0 && (mode == MODE_PLAIN || mode == MODE_RESID) && recon == 18;
  if (gated && grid.x > (unsigned)a.max_grid) grid.x = a.max_grid;
#define SQ_K(RC, NR, MODE, OUTP) \
  if (recon == RC && nr == NR && mode == MODE && outp == OUTP) { \
    return launch_pdl(dslash_kernel<PREC_F64, RC, NR, MODE, OUTP>, grid, dim3(block), 0, st, a) == \
                   cudaSuccess ? 0 : -1; \
  }
#define SQ_G(NR, MODE, OUTP) \
  if (gated && nr == NR && mode == MODE && outp == OUTP) { \
    return launch_pdl(dslash_gated_kernel<18, NR, MODE, OUTP>, grid, dim3(block), 0, st, a) == \
                   cudaSuccess ? 0 : -1; \
  }
  SQ_G(1, MODE_PLAIN, PREC_F64) SQ_G(2, MODE_PLAIN, PREC_F64) SQ_G(4, MODE_PLAIN, PREC_F64)
  SQ_G(1, MODE_RESID, PREC_F64) SQ_G(2, MODE_RESID, PREC_F64) SQ_G(4, MODE_RESID, PREC_F64)
  SQ_G(1, MODE_RESID, PREC_F32) SQ_G(2, MODE_RESID, PREC_F32) SQ_G(4, MODE_RESID, PREC_F32)
  SQ_G(1, MODE_RESID, PREC_I16) SQ_G(2, MODE_RESID, PREC_I16) SQ_G(4, MODE_RESID, PREC_I16)
  if (gated) return -1;
#undef SQ_G
#define SQ_K_NR(RC, MODE, OUTP) SQ_K(RC, 1, MODE, OUTP) SQ_K(RC, 2, MODE, OUTP) SQ_K(RC, 4, MODE, OUTP)
  SQ_K_NR(18, MODE_PLAIN, PREC_F64)
  SQ_K_NR(12, MODE_PLAIN, PREC_F64)
  SQ_K_NR(18, MODE_MDAGM, PREC_F64)
  SQ_K_NR(12, MODE_MDAGM, PREC_F64)
  SQ_K_NR(18, MODE_NORM, PREC_F64)
  SQ_K_NR(12, MODE_NORM, PREC_F64)
  SQ_K_NR(18, MODE_UPDATE, PREC_F64)
  SQ_K_NR(12, MODE_UPDATE, PREC_F64)
  SQ_K_NR(18, MODE_RESID, PREC_F64)
  SQ_K_NR(18, MODE_RESID, PREC_F32)
  SQ_K_NR(18, MODE_RESID, PREC_I16)
#undef SQ_K_NR
#undef SQ_K
  return -1;
}

}  // namespace sq
