// Host-side state of the library: the context, gauge fields, CG workspaces.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "../../include/sq.h"
#include "dslash.cuh"
#include "sq_kernels.h"
#include "sq_types.h"

namespace sq {

struct ServeEngine;
struct Tuner;

#define SQ_CUDA_TRY(expr)                                 \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) {                              \
      sq::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return _e == cudaErrorMemoryAllocation ? SQ_ERR_OOM : SQ_ERR_CUDA; \
    }                                                     \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Lattice extents all even and >= 2, volume <= 2^30: SQ_OK and *vol, else
// SQ_ERR_ARG.
int check_lattice_dims(const int dims[4], long *vol);

struct GaugeField {
  int id = 0;
  Geom g{};
  double long_s = 0;         // common scale s of the long links (det L = s^3)
  bool recon12_ok = false;   // long links are s * SU(3) to 1e-10 relative
  float fat_scale = 0, long_scale = 0;  // 16-bit global scales (max |element|)
  void *links[3][2][2] = {};            // [prec][recon 18 / 12][output parity]
  size_t bytes = 0;
  void *tmp[3] = {};                    // odd-parity temporaries for mdagm_apply
  std::atomic<int> users{0};

  bool has(int prec, int recon) const {
    return links[prec][recon == 12][0] != nullptr;
  }
  const char *link_ptr(int prec, int recon, int parity) const {
    return static_cast<const char *>(links[prec][recon == 12][parity]);
  }
  LinkScales scales(int prec, int recon) const;
};

struct sq_ctx_impl;

}  // namespace sq

struct sq_ctx {
  int device = 0;
  int sms = 0;                                       // multiprocessors of the device
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t in_use = 0;
  std::mutex mu;                                     // registry, budget
  std::map<int, std::unique_ptr<sq::GaugeField>> gauges;
  int next_gauge_id = 1;
  std::atomic<uint64_t> launches{0};
  sq::Tuner *tuner = nullptr;
  sq::ServeEngine *serve = nullptr;
  std::mutex solve_mu;                               // one blocking solve at a time

  int alloc(size_t bytes, void **p);
  void release(void *p, size_t bytes);
  sq::GaugeField *gauge(int id);
};

namespace sq {

// Dslash block size / RHS tile, chosen by the tuner (defaults before tuning).
struct DslashConfig {
  int block = 256;
  int nr = 1;
};

DslashConfig tuned_dslash(sq_ctx *ctx, const GaugeField &gf, int prec, int recon, int nrhs,
                          int mode, cudaStream_t st);
Tuner *tuner_create();
void tuner_destroy(Tuner *);

// Workspace and driver of a batched (nrhs >= 1) mixed-precision CG.
struct CGWork {
  sq_ctx *ctx = nullptr;
  GaugeField *gf = nullptr;
  int prec = PREC_F32, recon = 18, nrhs = 1;
  size_t f64_fb = 0, fb = 0;
  char *x64 = nullptr, *b64 = nullptr, *t64 = nullptr;
  char *r = nullptr, *p = nullptr, *t = nullptr;
  char *xs = nullptr;       // solution increment since the last reliable update
  size_t xs_fb = 0;
  SlotState *slots_d = nullptr, *slots_h = nullptr;
  double *partial = nullptr;
  unsigned *counters = nullptr;
  size_t bytes = 0;
  size_t partial_stride = 0;  // doubles per reduction region
  size_t counter_stride = 0;  // ticket counters per reduction region
  cudaGraphExec_t exec = nullptr;
  int exec_iters = 0;
  int exec_kernels = 0;       // kernels per replay
  DslashConfig cfg_norm, cfg_update, cfg_ru_plain, cfg_ru_resid;

  ~CGWork();
};

int cg_work_create(sq_ctx *ctx, GaugeField *gf, int prec, int recon, int nrhs, CGWork **out);
// Per-slot setup (host copy; upload with cg_slots_upload).
void cg_slot_setup(CGWork *w, int slot, double mass, double tol, double delta, int max_iter);
int cg_slots_upload(CGWork *w, cudaStream_t st);
int cg_slots_download(CGWork *w, cudaStream_t st);
// Launch sequences.
int cg_enqueue_init(CGWork *w, int guess, cudaStream_t st);
int cg_enqueue_ru(CGWork *w, cudaStream_t st);
int cg_enqueue_xpay(CGWork *w, cudaStream_t st);
// Reliable updates may follow every RU_PERIOD-th iteration (a checkpoint).
constexpr int RU_PERIOD = 4;
int cg_enqueue_iteration(CGWork *w, cudaStream_t st, int checkpoint);
// k iterations: a CUDA graph replay (captured on first use) or direct launches.
int cg_enqueue_block(CGWork *w, int k, bool graph, cudaStream_t st);
// Run until no slot is running; host polls the slot state after each block.
int cg_run(CGWork *w, int block_iters, bool graph, cudaStream_t st);
int slot_status_to_sq(int slot_status);
inline bool cg_slot_live(int s) { return s == SLOT_RUNNING || s == SLOT_WAIT || s == SLOT_INIT; }
void drop_multishift_works(const sq_ctx *ctx, int gauge_id);  // gauge_id < 0: all
void fill_stats(const SlotState &s, double seconds, long vh, sq_cg_stats *st);
// The launch shapes of the workspace's two sloppy Dslash kernels.
void fill_launch_stats(const CGWork *w, sq_cg_stats *st);

}  // namespace sq
