// Instantiations of the Dslash kernel family for PREC_F32 links and vectors.
#include "dslash.cuh"
#include "sq_kernels.h"

namespace sq {

int launch_dslash_f32(int recon, int nr, int mode, int outp, const DslashArgs &a, int block,
                       cudaStream_t st) {
  dim3 grid(((a.g.vh + block - 1) / block) * ((a.nrhs + nr - 1) / nr));
  const size_t smem = dslash_smem_bytes(PREC_F32, recon, nr, block);
  // the staged tiles take more than the default 48 KB of dynamic shared
  // memory: raise each kernel's limit once
#define SQ_K(RC, NR, MODE, OUTP) \
  if (recon == RC && nr == NR && mode == MODE && outp == OUTP) { \
    auto kern = dslash_kernel<PREC_F32, RC, NR, MODE, OUTP>; \
    if (NR > 1) { \
      static const cudaError_t attr_rc = cudaFuncSetAttribute( \
          kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
          (int)dslash_smem_bytes(PREC_F32, RC, NR, DslashBounds<PREC_F32, NR>::threads)); \
      if (attr_rc != cudaSuccess) return -1; \
    } \
    return launch_pdl(kern, grid, dim3(block), smem, st, a) == cudaSuccess ? 0 : -1; \
  }
#define SQ_K_NR(RC, MODE, OUTP) SQ_K(RC, 1, MODE, OUTP) SQ_K(RC, 2, MODE, OUTP) SQ_K(RC, 4, MODE, OUTP)
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
