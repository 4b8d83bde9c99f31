// The C ABI (include/sq.h): contexts, gauge fields, operators and solvers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <tuple>
#include <vector>

#include "gauge_pack.h"
#include "serve.h"
#include "sq_host.h"

using namespace sq;

namespace sq {

static thread_local char g_last_error[256] = "";

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what,
                file, line);
}

LinkScales GaugeField::scales(int prec, int recon) const {
  LinkScales s;
  s.keep = 0;
  s.fat_k = fat_scale / 32767.f;
  s.long_k = long_scale / 32767.f;
  s.recon_d = (long_s != 0) ? 1.0 / long_s : 0.0;
  s.recon_f = (float)s.recon_d;
  if (prec == PREC_I16 && recon == 12) s.recon_f = (float)((double)s.long_k / long_s);
  return s;
}

}  // namespace sq

int sq_ctx::alloc(size_t bytes, void **p) {
  {
    std::lock_guard<std::mutex> lk(mu);
    if (in_use + bytes > budget) return SQ_ERR_OOM;
    in_use += bytes;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    in_use -= bytes;
    *p = nullptr;
    set_last_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
    return e == cudaErrorMemoryAllocation ? SQ_ERR_OOM : SQ_ERR_CUDA;
  }
  return SQ_OK;
}

void sq_ctx::release(void *p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  std::lock_guard<std::mutex> lk(mu);
  in_use -= bytes;
}

GaugeField *sq_ctx::gauge(int id) {
  std::lock_guard<std::mutex> lk(mu);
  auto it = gauges.find(id);
  return it == gauges.end() ? nullptr : it->second.get();
}

// ------------------------------------------------------------------ helpers

namespace {

struct SolveCacheKey {
  int gid, prec, recon, nrhs;
  bool operator<(const SolveCacheKey &o) const {
    return std::tie(gid, prec, recon, nrhs) < std::tie(o.gid, o.prec, o.recon, o.nrhs);
  }
};

// Blocking-solve workspaces kept per context (graph and buffers reused).
struct SolveCache {
  std::map<SolveCacheKey, std::unique_ptr<CGWork>> works;
  void *staging = nullptr;  // canonical FP64 staging for host inputs/outputs
  size_t staging_bytes = 0;
};

std::mutex g_cache_mu;
std::map<const sq_ctx *, SolveCache> g_cache;

void drop_gauge_works(const sq_ctx *ctx, int gid) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto &c = g_cache[ctx];
  for (auto it = c.works.begin(); it != c.works.end();) {
    if (it->first.gid == gid) it = c.works.erase(it);
    else ++it;
  }
}

bool finite_all(const double *p, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

}  // namespace

// ------------------------------------------------------------------ context

extern "C" int sq_create(sq_ctx **out, int device, size_t hbm_budget_bytes) {
  if (!out) return SQ_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) return SQ_ERR_CUDA;
  if (device < 0 || device >= n) return SQ_ERR_ARG;
  SQ_CUDA_TRY(cudaSetDevice(device));
  std::unique_ptr<sq_ctx> c(new sq_ctx());
  c->device = device;
  SQ_CUDA_TRY(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
  SQ_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  size_t fr = 0, tot = 0;
  SQ_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  c->tuner = tuner_create();
  *out = c.release();
  return SQ_OK;
}

extern "C" int sq_destroy(sq_ctx *ctx) {
  if (!ctx) return SQ_ERR_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->serve) {
    serve_shutdown(ctx->serve);
    ctx->serve = nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(ctx);
    if (it != g_cache.end()) {
      it->second.works.clear();
      if (it->second.staging) cudaFree(it->second.staging);
      g_cache.erase(it);
    }
  }
  drop_multishift_works(ctx, -1);
  std::vector<int> ids;
  for (auto &kv : ctx->gauges) ids.push_back(kv.first);
  for (int id : ids) gauge_free(ctx, id);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  tuner_destroy(ctx->tuner);
  delete ctx;
  return SQ_OK;
}

extern "C" const char *sq_strerror(int s) {
  switch (s) {
    case SQ_OK: return "ok";
    case SQ_PENDING: return "pending";
    case SQ_NOT_CONVERGED: return "not converged (max_iter reached)";
    case SQ_ERR_ARG: return "invalid argument";
    case SQ_ERR_OOM: return "out of device memory or HBM budget";
    case SQ_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case SQ_ERR_NONFINITE: return "non-finite value";
    case SQ_ERR_TIMEOUT: return "timeout";
    case SQ_ERR_BUSY: return "busy";
    case SQ_ERR_NOTFOUND: return "not found";
    case SQ_ERR_UNSUPPORTED: return "unsupported combination";
  }
  return "unknown status";
}

extern "C" void sq_cg_opts_default(sq_cg_opts *o) {
  if (!o) return;
  o->precision = SQ_PREC_F32;
  o->long_recon = 18;
  o->delta = -1.0;  // precision default: 0.001 (FP32), 0.1 (16-bit)
  o->max_iter = 100000;
  o->block_iters = 16;
  o->flags = 0;
  o->stream = nullptr;
}

extern "C" uint64_t sq_kernel_launches(const sq_ctx *ctx) {
  return ctx ? ctx->launches.load() : 0;
}

// --------------------------------------------------------------------- gauge

extern "C" int gauge_load(sq_ctx *ctx, const int dims[4], const double *fat, const double *lng,
                          unsigned flags, int *gauge_id) {
  if (!ctx || !dims || !fat || !lng || !gauge_id) return SQ_ERR_ARG;
  long vol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || (dims[mu] & 1)) return SQ_ERR_ARG;
    vol *= dims[mu];
    if (vol > (1L << 30)) return SQ_ERR_ARG;
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  std::unique_ptr<GaugeField> gf(new GaugeField());
  Geom &g = gf->g;
  for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
  g.st[0] = 1;
  g.st[1] = dims[0];
  g.st[2] = dims[0] * dims[1];
  g.st[3] = dims[0] * dims[1] * dims[2];
  g.lxh = dims[0] / 2;
  g.vh = (int)(vol / 2);
  g.stride = (g.vh + 63) / 64 * 64;
  g.nchunks = (g.vh + CHUNK - 1) / CHUNK;
  g.nwchunks = (g.vh + 31) / 32;
  g.ngroups = (g.nwchunks + 31) / 32;
  g.t_antiperiodic = (flags & SQ_GAUGE_ANTIPERIODIC_T) ? 1 : 0;
  geom_set_divisor(g, 0, (uint32_t)g.lxh);
  geom_set_divisor(g, 1, (uint32_t)dims[1]);
  geom_set_divisor(g, 2, (uint32_t)dims[2]);

  const size_t nlink_bytes = (size_t)vol * 4 * 9 * 16;
  const double *dfat = fat, *dlng = lng;
  void *tmp = nullptr;
  int rc;
  double l0[18];
  if (!(flags & SQ_GAUGE_DEVICE_PTRS)) {
    if (!finite_all(fat, (size_t)vol * 72) || !finite_all(lng, (size_t)vol * 72))
      return SQ_ERR_NONFINITE;
    // staging of the canonical links, freed before return: outside the budget
    cudaError_t ae = cudaMalloc(&tmp, 2 * nlink_bytes);
    if (ae != cudaSuccess) {
      set_last_cuda_error(ae, "cudaMalloc(link staging)", __FILE__, __LINE__);
      return SQ_ERR_OOM;
    }
    dfat = static_cast<double *>(tmp);
    dlng = dfat + (size_t)vol * 72;
    cudaMemcpyAsync((void *)dfat, fat, nlink_bytes, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void *)dlng, lng, nlink_bytes, cudaMemcpyHostToDevice, st);
    std::memcpy(l0, lng, sizeof(l0));
  } else {
    if (cudaMemcpyAsync(l0, lng, sizeof(l0), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SQ_ERR_ARG;
  }
  // common scale of the long links from det L(0) = s^3
  {
    auto C = [&](int r, int c) { return std::complex<double>(l0[2 * (3 * r + c)], l0[2 * (3 * r + c) + 1]); };
    std::complex<double> det = C(0, 0) * (C(1, 1) * C(2, 2) - C(1, 2) * C(2, 1)) -
                               C(0, 1) * (C(1, 0) * C(2, 2) - C(1, 2) * C(2, 0)) +
                               C(0, 2) * (C(1, 0) * C(2, 1) - C(1, 1) * C(2, 0));
    gf->long_s = std::cbrt(det.real());
    if (std::abs(det.imag()) > 1e-10 * std::abs(det) || gf->long_s == 0) gf->long_s = 0;
  }
  unsigned long long *stats_d = nullptr;
  unsigned long long stats_h[3] = {0, 0, 0};
  cudaError_t e = cudaMalloc(&stats_d, sizeof(stats_h));
  if (e == cudaSuccess) {
    cudaMemsetAsync(stats_d, 0, sizeof(stats_h), st);
    launch_gauge_stats(dfat, dlng, vol * 4, gf->long_s != 0 ? 1.0 / gf->long_s : 0.0, stats_d, st);
    ctx->launches++;
    cudaMemcpyAsync(stats_h, stats_d, sizeof(stats_h), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    cudaFree(stats_d);
  }
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "gauge statistics", __FILE__, __LINE__);
    if (tmp) cudaFree(tmp);
    return SQ_ERR_CUDA;
  }
  double fmax_, lmax_, rerr;
  std::memcpy(&fmax_, &stats_h[0], 8);
  std::memcpy(&lmax_, &stats_h[1], 8);
  std::memcpy(&rerr, &stats_h[2], 8);
  if (!std::isfinite(fmax_) || !std::isfinite(lmax_)) {
    if (tmp) cudaFree(tmp);
    return SQ_ERR_NONFINITE;
  }
  gf->fat_scale = (float)fmax_;
  gf->long_scale = (float)lmax_;
  gf->recon12_ok = gf->long_s != 0 && rerr <= 1e-10 * std::abs(gf->long_s);
  PackScales ps;
  ps.fat_inv = gf->fat_scale > 0 ? 32767.0f / gf->fat_scale : 0.f;
  ps.long_inv = gf->long_scale > 0 ? 32767.0f / gf->long_scale : 0.f;

  rc = SQ_OK;
  for (int prec = 0; prec < 3 && rc == SQ_OK; ++prec) {
    if (prec == PREC_F64 && (flags & SQ_GAUGE_NO_F64)) continue;
    if (prec == PREC_F32 && (flags & SQ_GAUGE_NO_F32)) continue;
    if (prec == PREC_I16 && (flags & SQ_GAUGE_NO_I16)) continue;
    for (int recon : {18, 12}) {
      if (recon == 12 && (!gf->recon12_ok || (flags & SQ_GAUGE_NO_LONG12))) continue;
      size_t b = link_site_bytes(prec, recon) * g.stride;
      for (int par = 0; par < 2 && rc == SQ_OK; ++par) {
        rc = ctx->alloc(b, &gf->links[prec][recon == 12][par]);
        if (rc == SQ_OK) gf->bytes += b;
      }
      if (rc) break;
      if (launch_gauge_pack(prec, recon, g, dfat, dlng, gf->links[prec][recon == 12][0],
                            gf->links[prec][recon == 12][1], ps, st) != 0)
        rc = SQ_ERR_ARG;
      ctx->launches++;
    }
  }
  e = cudaStreamSynchronize(st);
  if (tmp) cudaFree(tmp);
  if (rc == SQ_OK && e != cudaSuccess) {
    set_last_cuda_error(e, "gauge pack", __FILE__, __LINE__);
    rc = SQ_ERR_CUDA;
  }
  if (rc != SQ_OK) {
    for (auto &a : gf->links)
      for (auto &b : a)
        for (auto &p : b)
          if (p) cudaFree(p);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->in_use -= gf->bytes;
    return rc;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  gf->id = ctx->next_gauge_id++;
  *gauge_id = gf->id;
  ctx->gauges[gf->id] = std::move(gf);
  return SQ_OK;
}

extern "C" int gauge_free(sq_ctx *ctx, int gauge_id) {
  if (!ctx) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (ctx->serve && serve_uses_gauge(ctx->serve, gauge_id)) return SQ_ERR_BUSY;
  drop_gauge_works(ctx, gauge_id);
  drop_multishift_works(ctx, gauge_id);
  if (gf->users.load() > 0) return SQ_ERR_BUSY;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  size_t freed = gf->bytes;
  for (auto &a : gf->links)
    for (auto &b : a)
      for (auto &p : b)
        if (p) cudaFree(p);
  for (int k = 0; k < 3; ++k)
    if (gf->tmp[k]) {
      cudaFree(gf->tmp[k]);
      freed += spinor_bytes(k, gf->g.stride);
    }
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->in_use -= freed;
  ctx->gauges.erase(gauge_id);
  return SQ_OK;
}

extern "C" int sq_spinor_bytes(sq_ctx *ctx, int gauge_id, int prec, size_t *bytes, int *stride) {
  if (!ctx || prec < 0 || prec > 2) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (bytes) *bytes = spinor_bytes(prec, gf->g.stride);
  if (stride) *stride = gf->g.stride;
  return SQ_OK;
}

extern "C" int sq_pack_spinor(sq_ctx *ctx, int gauge_id, int prec, const double *canon_dev,
                              void *packed_dev, void *stream) {
  if (!ctx || !canon_dev || !packed_dev || prec < 0 || prec > 2) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  cudaSetDevice(ctx->device);
  if (launch_pack(prec, gf->g, canon_dev, 0, packed_dev, 0, 1, (cudaStream_t)stream))
    return SQ_ERR_ARG;
  ctx->launches++;
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}

extern "C" int sq_unpack_spinor(sq_ctx *ctx, int gauge_id, int prec, const void *packed_dev,
                                double *canon_dev, void *stream) {
  if (!ctx || !canon_dev || !packed_dev || prec < 0 || prec > 2) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  cudaSetDevice(ctx->device);
  if (launch_unpack(prec, gf->g, packed_dev, 0, canon_dev, 0, 1, (cudaStream_t)stream))
    return SQ_ERR_ARG;
  ctx->launches++;
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}

// ----------------------------------------------------------------- operators

extern "C" int dslash_apply(sq_ctx *ctx, int gauge_id, int out_parity, int prec, int long_recon,
                            const void *in_dev, void *out_dev, void *stream) {
  if (!ctx || !in_dev || !out_dev || in_dev == out_dev) return SQ_ERR_ARG;
  if (out_parity < 0 || out_parity > 1 || prec < 0 || prec > 2) return SQ_ERR_ARG;
  if (long_recon != 18 && long_recon != 12) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(prec, long_recon)) return SQ_ERR_UNSUPPORTED;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  DslashConfig cfg = tuned_dslash(ctx, *gf, prec, long_recon, 1, MODE_PLAIN, st);
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = gf->g;
  a.out_parity = out_parity;
  a.links = gf->link_ptr(prec, long_recon, out_parity);
  a.ls = gf->scales(prec, long_recon);
  a.in = static_cast<const char *>(in_dev);
  a.out = static_cast<char *>(out_dev);
  a.nrhs = 1;
  a.gate = GATE_NONE;
  if (launch_dslash(prec, long_recon, 1, MODE_PLAIN, prec, a, cfg.block, st)) return SQ_ERR_ARG;
  ctx->launches++;
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}

extern "C" int dslash_apply_multi(sq_ctx *ctx, int gauge_id, int out_parity, int prec,
                                  int long_recon, int nrhs, const void *in_dev, void *out_dev,
                                  void *stream) {
  if (!ctx || !in_dev || !out_dev || in_dev == out_dev) return SQ_ERR_ARG;
  if (out_parity < 0 || out_parity > 1 || prec < 0 || prec > 2) return SQ_ERR_ARG;
  if (long_recon != 18 && long_recon != 12) return SQ_ERR_ARG;
  if (nrhs < 1 || nrhs > 64) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(prec, long_recon)) return SQ_ERR_UNSUPPORTED;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  DslashConfig cfg = tuned_dslash(ctx, *gf, prec, long_recon, nrhs, MODE_PLAIN, st);
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = gf->g;
  a.out_parity = out_parity;
  a.links = gf->link_ptr(prec, long_recon, out_parity);
  a.ls = gf->scales(prec, long_recon);
  a.in = static_cast<const char *>(in_dev);
  a.out = static_cast<char *>(out_dev);
  a.in_fb = a.out_fb = spinor_bytes(prec, gf->g.stride);
  a.nrhs = nrhs;
  a.gate = GATE_NONE;
  if (launch_dslash(prec, long_recon, cfg.nr, MODE_PLAIN, prec, a, cfg.block, st))
    return SQ_ERR_ARG;
  ctx->launches++;
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}

extern "C" int sq_tuned_launch(sq_ctx *ctx, int gauge_id, int prec, int long_recon, int nrhs,
                               int mode, void *stream, int *block, int *rhs_tile) {
  if (!ctx || !block || !rhs_tile || prec < 0 || prec > 2) return SQ_ERR_ARG;
  if (long_recon != 18 && long_recon != 12) return SQ_ERR_ARG;
  if (nrhs < 1 || nrhs > 64) return SQ_ERR_ARG;
  if (mode != MODE_PLAIN && mode != MODE_MDAGM && mode != MODE_NORM && mode != MODE_UPDATE)
    return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(prec, long_recon)) return SQ_ERR_UNSUPPORTED;
  cudaSetDevice(ctx->device);
  DslashConfig cfg = tuned_dslash(ctx, *gf, prec, long_recon, nrhs, mode, (cudaStream_t)stream);
  *block = std::min(cfg.block, dslash_max_block(prec, cfg.nr));
  *rhs_tile = cfg.nr;
  return SQ_OK;
}

extern "C" int mdagm_apply(sq_ctx *ctx, int gauge_id, int prec, int long_recon, double mass,
                           const void *in_dev, void *out_dev, void *stream) {
  if (!ctx || !in_dev || !out_dev || in_dev == out_dev || prec < 0 || prec > 2) return SQ_ERR_ARG;
  if (long_recon != 18 && long_recon != 12) return SQ_ERR_ARG;
  if (!std::isfinite(mass)) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(prec, long_recon)) return SQ_ERR_UNSUPPORTED;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (!gf->tmp[prec]) {
    int rc = ctx->alloc(spinor_bytes(prec, gf->g.stride), &gf->tmp[prec]);
    if (rc) return rc;
  }
  DslashConfig cfg = tuned_dslash(ctx, *gf, prec, long_recon, 1, MODE_PLAIN, st);
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = gf->g;
  a.nrhs = 1;
  a.gate = GATE_NONE;
  a.ls = gf->scales(prec, long_recon);
  a.out_parity = 1;
  a.links = gf->link_ptr(prec, long_recon, 1);
  a.in = static_cast<const char *>(in_dev);
  a.out = static_cast<char *>(gf->tmp[prec]);
  if (launch_dslash(prec, long_recon, 1, MODE_PLAIN, prec, a, cfg.block, st)) return SQ_ERR_ARG;
  a.out_parity = 0;
  a.links = gf->link_ptr(prec, long_recon, 0);
  a.in = static_cast<const char *>(gf->tmp[prec]);
  a.out = static_cast<char *>(out_dev);
  a.p = static_cast<const char *>(in_dev);
  a.m2_const = mass * mass;
  if (launch_dslash(prec, long_recon, 1, MODE_MDAGM, prec, a, cfg.block, st)) return SQ_ERR_ARG;
  ctx->launches += 2;
  SQ_CUDA_TRY(cudaGetLastError());
  return SQ_OK;
}

// ------------------------------------------------------------------- solvers

namespace sq {

// Shared body of cg_solve / cg_solve_multi / the refinement of multi-shift;
// the caller holds ctx->solve_mu.
int solve_batch_locked(sq_ctx *ctx, int gauge_id, int nrhs, const double *src,
                       const double *masses, double tol, const sq_cg_opts *opts_in, double *x,
                       sq_cg_stats *stats) {
  if (!ctx || !src || !masses || !x || nrhs < 1 || nrhs > 64) return SQ_ERR_ARG;
  if (!(tol > 0) || !std::isfinite(tol)) return SQ_ERR_ARG;
  for (int k = 0; k < nrhs; ++k)
    if (!(masses[k] > 0) || !std::isfinite(masses[k])) return SQ_ERR_ARG;
  sq_cg_opts o;
  sq_cg_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (o.precision < 0 || o.precision > 2) return SQ_ERR_ARG;
  if (o.long_recon != 18 && o.long_recon != 12) return SQ_ERR_ARG;
  if (o.delta < 0) o.delta = (o.precision == PREC_I16) ? 0.1 : 0.001;
  if (o.max_iter < 1 || o.block_iters < 1 || !(o.delta >= 0) || o.delta >= 1) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(o.precision, o.long_recon)) return SQ_ERR_UNSUPPORTED;
  const bool dev = (o.flags & SQ_CG_DEVICE_PTRS) != 0;
  const bool guess = (o.flags & SQ_CG_INITIAL_GUESS) != 0;
  const size_t vec_elems = (size_t)3 * gf->g.vh;  // complex per vector
  // Non-finite sources are found on the device (|b|^2 of a system is then
  // not finite and the system ends SLOT_NONFINITE, i.e. SQ_ERR_NONFINITE,
  // without iterating), as for device pointers: a host pass over the
  // source would sit between the call and its first copy.

  cudaSetDevice(ctx->device);
  auto t0 = std::chrono::steady_clock::now();
  // Run on the caller's stream unless it is a default stream (those cannot
  // be captured into a graph); then the context's stream, after the caller's.
  cudaStream_t st = ctx->stream;
  cudaStream_t user = (cudaStream_t)o.stream;
  if (user == cudaStreamLegacy || user == cudaStreamPerThread) user = nullptr;
  if (user) st = user;
  else  // a default stream (NULL: the legacy one): the caller's work on it first
    SQ_CUDA_TRY(cudaStreamSynchronize(o.stream ? (cudaStream_t)o.stream : cudaStreamLegacy));

  CGWork *w = nullptr;
  SolveCache *cache;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache = &g_cache[ctx];
    SolveCacheKey key{gauge_id, o.precision, o.long_recon, nrhs};
    auto it = cache->works.find(key);
    if (it != cache->works.end()) w = it->second.get();
  }
  if (!w) {
    int rc = cg_work_create(ctx, gf, o.precision, o.long_recon, nrhs, &w);
    if (rc) return rc;
    w->cfg_norm = tuned_dslash(ctx, *gf, o.precision, o.long_recon, nrhs, MODE_NORM, st);
    w->cfg_update = tuned_dslash(ctx, *gf, o.precision, o.long_recon, nrhs, MODE_UPDATE, st);
    w->cfg_ru_plain = tuned_dslash(ctx, *gf, PREC_F64, 18, nrhs, MODE_PLAIN, st);
    w->cfg_ru_resid = w->cfg_ru_plain;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache->works[SolveCacheKey{gauge_id, o.precision, o.long_recon, nrhs}].reset(w);
  }
  // staging for host pointers
  const size_t canon_bytes = vec_elems * 16 * nrhs;
  double *csrc = const_cast<double *>(src), *cx = x;
  if (!dev) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (cache->staging_bytes < canon_bytes) {
      if (cache->staging) ctx->release(cache->staging, cache->staging_bytes);
      cache->staging = nullptr;
      cache->staging_bytes = 0;
      int rc = ctx->alloc(canon_bytes, &cache->staging);
      if (rc) return rc;
      cache->staging_bytes = canon_bytes;
    }
    csrc = cx = static_cast<double *>(cache->staging);
    SQ_CUDA_TRY(cudaMemcpyAsync(csrc, src, canon_bytes, cudaMemcpyHostToDevice, st));
  }
  if (launch_pack(PREC_F64, gf->g, csrc, vec_elems, w->b64, w->f64_fb, nrhs, st)) return SQ_ERR_ARG;
  ctx->launches++;
  if (guess) {
    if (!dev) SQ_CUDA_TRY(cudaMemcpyAsync(cx, x, canon_bytes, cudaMemcpyHostToDevice, st));
    if (launch_pack(PREC_F64, gf->g, cx, vec_elems, w->x64, w->f64_fb, nrhs, st)) return SQ_ERR_ARG;
    ctx->launches++;
  }
  for (int k = 0; k < nrhs; ++k) cg_slot_setup(w, k, masses[k], tol, o.delta, o.max_iter);
  int rc;
  if ((rc = cg_slots_upload(w, st))) return rc;
  if ((rc = cg_enqueue_init(w, guess ? 1 : 0, st))) return rc;
  if ((rc = cg_run(w, o.block_iters, !(o.flags & SQ_CG_NO_GRAPH), st))) return rc;
  if (launch_unpack(PREC_F64, gf->g, w->x64, w->f64_fb, cx, vec_elems, nrhs, st)) return SQ_ERR_ARG;
  ctx->launches++;
  if (!dev) SQ_CUDA_TRY(cudaMemcpyAsync(x, cx, canon_bytes, cudaMemcpyDeviceToHost, st));
  SQ_CUDA_TRY(cudaStreamSynchronize(st));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int first_err = SQ_OK;
  bool not_conv = false;
  for (int k = 0; k < nrhs; ++k) {
    if (stats) {
      fill_stats(w->slots_h[k], secs, gf->g.vh, stats + k);
      fill_launch_stats(w, stats + k);
    }
    int s = slot_status_to_sq(w->slots_h[k].status);
    if (s < 0 && first_err == SQ_OK) first_err = s;
    if (s == SQ_NOT_CONVERGED) not_conv = true;
  }
  return first_err != SQ_OK ? first_err : not_conv ? SQ_NOT_CONVERGED : SQ_OK;
}

int solve_batch(sq_ctx *ctx, int gauge_id, int nrhs, const double *src, const double *masses,
                double tol, const sq_cg_opts *opts, double *x, sq_cg_stats *stats) {
  if (!ctx) return SQ_ERR_ARG;
  std::lock_guard<std::mutex> solve_lock(ctx->solve_mu);
  return solve_batch_locked(ctx, gauge_id, nrhs, src, masses, tol, opts, x, stats);
}

}  // namespace sq

extern "C" int cg_solve(sq_ctx *ctx, int gauge_id, const double *src_even, double mass, double tol,
                        const sq_cg_opts *opts, double *x_even, sq_cg_stats *stats) {
  return solve_batch(ctx, gauge_id, 1, src_even, &mass, tol, opts, x_even, stats);
}

extern "C" int cg_solve_multi(sq_ctx *ctx, int gauge_id, int nrhs, const double *src,
                              const double *masses, double tol, const sq_cg_opts *opts, double *x,
                              sq_cg_stats *stats) {
  return solve_batch(ctx, gauge_id, nrhs, src, masses, tol, opts, x, stats);
}
