// Host interface of the gauge-field pack kernels.
#pragma once

#include <cuda_runtime.h>

#include "sq_types.h"

namespace sq {

struct PackScales {
  float fat_inv;   // 32767 / fat scale (FP32): 16-bit code = rint(v * fat_inv)
  float long_inv;  // 32767 / long scale
};

// Per-field maxima over nlinks = 4V links: out[0] = max |re|,|im| of fat,
// out[1] = same for long, out[2] = max deviation of the long links' third row
// from inv_s * conj(row0 x row1).  out holds non-negative doubles as u64 bits
// and must be zeroed by the caller.
int launch_gauge_stats(const double *fat, const double *lng, long nlinks, double inv_s,
                       unsigned long long *out, cudaStream_t st);

int launch_gauge_pack(int prec, int recon, const Geom &g, const double *fat, const double *lng,
                      void *links_even, void *links_odd, const PackScales &ps, cudaStream_t st);

// Bytes per site (16 hop matrices) of one parity's links in a layout.
size_t link_site_bytes(int prec, int recon);

}  // namespace sq
