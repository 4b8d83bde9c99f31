// Dispatch of a Dslash launch to the per-precision instantiation files.
#include "dslash.cuh"

namespace sq {

int launch_dslash_f64(int, int, int, int, const DslashArgs &, int, cudaStream_t);
int launch_dslash_f32(int, int, int, int, const DslashArgs &, int, cudaStream_t);
int launch_dslash_i16(int, int, int, int, const DslashArgs &, int, cudaStream_t);

int launch_dslash(int prec, int recon, int nr, int mode, int outp, const DslashArgs &a,
                  int block, cudaStream_t stream) {
  if (a.g.vh <= 0) return 0;
  // whole warps (the kernels' sums are per warp of 32 sites), at most 512
  if (block <= 0 || block % 32 != 0 || block > 512) return -1;
  const int cap = dslash_max_block(prec, nr);
  if (block > cap) block = cap;
  switch (prec) {
    case PREC_F64: return launch_dslash_f64(recon, nr, mode, outp, a, block, stream);
    case PREC_F32: return launch_dslash_f32(recon, nr, mode, outp, a, block, stream);
    case PREC_I16: return launch_dslash_i16(recon, nr, mode, outp, a, block, stream);
  }
  return -1;
}

}  // namespace sq
