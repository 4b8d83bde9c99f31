// mdagm_apply_static: the normal operator m^2 - D_eo D_oe (the same two Dslash
// kernels as mdagm_apply) with its odd-parity temporary in a fixed device
// array owned by this library, so that a call allocates nothing.
//
// Who needs it: callers that cannot let the library allocate device memory
// at call time -- applications that reserve all of HBM up front through
// their own allocator or memory pool and forbid libraries to allocate behind
// it, and latency-critical loops where a first-use cudaMalloc would be an
// unpredictable stall.  mdagm_apply, by contrast, allocates its temporary on
// first use per gauge field and precision.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds SQ_STATIC_SCRATCH_BYTES of it until the process
// exits.  In host code its name is only a host-side stand-in, never a device
// address, so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels as a plain pointer.
#include <cmath>
#include <cstring>
#include <mutex>

#include "sq_host.h"

namespace {

static __device__ __align__(256) unsigned char g_mdagm_scratch[SQ_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current device), looked
// up on the first call for that device (a one-time set-up: that first call
// should come before any stream capture).
int scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return SQ_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_mdagm_scratch);
    if (e != cudaSuccess || p == nullptr) {
      sq::set_last_cuda_error(e, "cudaGetSymbolAddress(static scratch)", __FILE__, __LINE__);
      return SQ_ERR_CUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return SQ_OK;
}

}  // namespace

using namespace sq;

extern "C" int mdagm_apply_static(sq_ctx *ctx, int gauge_id, int prec, int long_recon,
                                  double mass, const void *in_dev, void *out_dev, void *stream) {
  if (!ctx || !in_dev || !out_dev || in_dev == out_dev || prec < 0 || prec > 2) return SQ_ERR_ARG;
  if (long_recon != 18 && long_recon != 12) return SQ_ERR_ARG;
  if (!std::isfinite(mass)) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(prec, long_recon)) return SQ_ERR_UNSUPPORTED;
  // the odd-parity temporary must fit the fixed array
  if (spinor_bytes(prec, gf->g.stride) > (size_t)SQ_STATIC_SCRATCH_BYTES) return SQ_ERR_ARG;
  SQ_CUDA_TRY(cudaSetDevice(ctx->device));
  void *tmp = nullptr;
  int rc = scratch_address(ctx->device, &tmp);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int block = 256;  // fixed: the launch-shape tuner allocates while it times
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = gf->g;
  a.nrhs = 1;
  a.gate = GATE_NONE;
  a.ls = gf->scales(prec, long_recon);
  a.out_parity = 1;
  a.links = gf->link_ptr(prec, long_recon, 1);
  a.in = static_cast<const char *>(in_dev);
  a.out = static_cast<char *>(tmp);
  if (launch_dslash(prec, long_recon, 1, MODE_PLAIN, prec, a, block, st)) return SQ_ERR_ARG;
  a.out_parity = 0;
  a.links = gf->link_ptr(prec, long_recon, 0);
  a.in = static_cast<const char *>(tmp);
  a.out = static_cast<char *>(out_dev);
  a.p = static_cast<const char *>(in_dev);
  a.m2_const = mass * mass;
  if (launch_dslash(prec, long_recon, 1, MODE_MDAGM, prec, a, block, st)) return SQ_ERR_ARG;
  ctx->launches += 2;
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}
