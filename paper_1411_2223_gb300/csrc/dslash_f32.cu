// Instantiations of the Dslash kernel family for PREC_F32 links and vectors.
#include "dslash.cuh"
#include "sq_kernels.h"

namespace sq {

int launch_dslash_f32(int recon, int nr, int mode, int outp, const DslashArgs &a, int block,
                       cudaStream_t st) {
  dim3 grid(((a.g.vh + block - 1) / block) * ((a.nrhs + nr - 1) / nr));
#define SQ_K(RC, NR, MODE, OUTP) \
  if (recon == RC && nr == NR && mode == MODE && outp == OUTP) { \
    return launch_pdl(dslash_kernel<PREC_F32, RC, NR, MODE, OUTP>, grid, dim3(block), 0, st, a) == \
                   cudaSuccess ? 0 : -1; \
  }
#define SQ_K_NR(RC, MODE, OUTP) SQ_K(RC, 1, MODE, OUTP) SQ_K(RC, 2, MODE, OUTP) SQ_K(RC, 4, MODE, OUTP) \
  SQ_K(RC, 6, MODE, OUTP) SQ_K(RC, 8, MODE, OUTP) SQ_K(RC, 12, MODE, OUTP)
  SQ_K_NR(18, MODE_PLAIN, PREC_F32)
  SQ_K_NR(12, MODE_PLAIN, PREC_F32)
  SQ_K_NR(18, MODE_MDAGM, PREC_F32)
  SQ_K_NR(12, MODE_MDAGM, PREC_F32)
  SQ_K_NR(18, MODE_NORM, PREC_F32)
  SQ_K_NR(12, MODE_NORM, PREC_F32)
  SQ_K_NR(18, MODE_UPDATE, PREC_F32)
  SQ_K_NR(12, MODE_UPDATE, PREC_F32)
#undef SQ_K_NR
#undef SQ_K
  return -1;
}

}  // namespace sq
