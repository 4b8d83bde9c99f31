// Run-time autotuner of the Dslash launch shape: threads per block and the
// number of right-hand sides each thread applies a loaded link to.  The
// paper's QUDA path picks launch parameters "dynamically and automatically"
// (Sec. 3); this tuner times every candidate with CUDA events on the first
// use of a (lattice, precision, link format, batch size) key and caches the
// winner for the context.  SQ_TUNE_CACHE=<file> persists the cache across
// processes.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "sq_host.h"

namespace sq {

struct Tuner {
  std::mutex mu;
  std::map<std::string, DslashConfig> cache;
  std::string path;
};

static std::string tune_key(const Geom &g, int prec, int recon, int nrhs, int mode) {
  std::ostringstream s;
  s << "dslash_v3:" << g.L[0] << "x" << g.L[1] << "x" << g.L[2] << "x" << g.L[3] << ":p" << prec
    << ":r" << recon << ":n" << nrhs << ":m" << mode;
  return s.str();
}

Tuner *tuner_create() {
  Tuner *t = new Tuner();
  const char *p = std::getenv("SQ_TUNE_CACHE");
  if (p && *p) {
    t->path = p;
    std::ifstream in(t->path);
    std::string key;
    DslashConfig c;
    while (in >> key >> c.block >> c.nr) t->cache[key] = c;
  }
  return t;
}

void tuner_destroy(Tuner *t) { delete t; }

static void tuner_save(Tuner *t) {
  if (t->path.empty()) return;
  std::ofstream out(t->path);
  for (auto &kv : t->cache) out << kv.first << " " << kv.second.block << " " << kv.second.nr << "\n";
}

DslashConfig tuned_dslash(sq_ctx *ctx, const GaugeField &gf, int prec, int recon, int nrhs,
                          int mode, cudaStream_t st) {
  // PLAIN and the reduction epilogues (MDAGM, NORM, UPDATE) are tuned apart:
  // a reduction favours more, smaller blocks per SM.  RESID uses the PLAIN
  // shape.
  if (mode != MODE_MDAGM && mode != MODE_NORM && mode != MODE_UPDATE) mode = MODE_PLAIN;
  const bool reduces = mode != MODE_PLAIN;
  DslashConfig def;
  def.block = 256;
  def.nr = nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1;
  Tuner *t = ctx->tuner;
  if (!t || !gf.has(prec, recon)) return def;
  const std::string key = tune_key(gf.g, prec, recon, nrhs, mode);
  std::lock_guard<std::mutex> lk(t->mu);
  auto it = t->cache.find(key);
  if (it != t->cache.end()) return it->second;
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return def;

  const Geom &g = gf.g;
  size_t fb = spinor_bytes(prec, g.stride);
  void *in = nullptr, *out = nullptr, *aux = nullptr;
  // aux: p field, slot states, partial sums, the ticket counters and (UPDATE)
  // the solution increment xs
  const size_t xs_b = spinor_bytes(xs_prec(prec), g.stride) * nrhs;
  size_t aux_b = fb * nrhs + sizeof(SlotState) * nrhs + sizeof(double) * nrhs * red_stride(g) +
                 sizeof(unsigned) * nrhs * ticket_stride(g) + 256 + xs_b;
  if (cudaMalloc(&in, fb * nrhs) != cudaSuccess) return def;
  if (cudaMalloc(&out, fb * nrhs) != cudaSuccess || cudaMalloc(&aux, aux_b) != cudaSuccess) {
    cudaFree(in);
    if (out) cudaFree(out);
    return def;
  }
  cudaMemsetAsync(in, 0, fb * nrhs, st);
  cudaMemsetAsync(aux, 0, aux_b, st);
  char *auxc = static_cast<char *>(aux);
  SlotState *slots = reinterpret_cast<SlotState *>(auxc + fb * nrhs);
  double *partial = reinterpret_cast<double *>(slots + nrhs);
  unsigned *counter = reinterpret_cast<unsigned *>(partial + (size_t)nrhs * red_stride(g));
  // xs at the end, 256-byte aligned: rounding the offset down stays inside
  // the 256 spare bytes after the counters
  char *xs = auxc + (aux_b - xs_b) / 256 * 256;
  if (reduces) {
    // running systems that the timed launches cannot stop (an UPDATE epilogue
    // never sees convergence or max_iter)
    std::vector<SlotState> hs(nrhs);
    for (auto &s : hs) {
      std::memset(&s, 0, sizeof(s));
      s.status = SLOT_RUNNING;
      s.m2 = 1e-4;
      s.rr = 1.0;
      s.tol2b2 = -1.0;
      s.max_iter = 1 << 30;
    }
    cudaMemcpyAsync(slots, hs.data(), sizeof(SlotState) * nrhs, cudaMemcpyHostToDevice, st);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  DslashArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.out_parity = 1;
  a.links = gf.link_ptr(prec, recon, 1);
  a.ls = gf.scales(prec, recon);
  a.in = static_cast<const char *>(in);
  a.out = static_cast<char *>(out);
  a.in_fb = a.out_fb = fb;
  a.nrhs = nrhs;
  a.gate = GATE_NONE;
  if (reduces) {
    a.slots = slots;
    a.partial = partial;
    a.counter = counter;
    a.gate = GATE_RUNNING;
  }
  if (mode == MODE_MDAGM || mode == MODE_UPDATE) {
    a.out_parity = 0;
    a.links = gf.link_ptr(prec, recon, 0);
    a.p = auxc;
    a.p_fb = fb;
  }
  if (mode == MODE_UPDATE) {
    a.xs = xs;
    a.xs_fb = spinor_bytes(xs_prec(prec), g.stride);
    a.xs_prec = xs_prec(prec);
  }
  // RHS tiles; the many-RHS tiles (8, 12) exist for the FP32 kernels only
  // (launch_dslash refuses the others and the candidate is skipped)
  std::vector<int> nrs = {1};
  for (int nr : {2, 4, 8, 12})
    if (nrhs >= nr) nrs.push_back(nr);
  float best = 1e30f;
  DslashConfig best_c = def;
  const int reps = 5;
  for (int nr : nrs) {
    const int max_block = dslash_max_block(prec, nr);
    for (int block = 128; block <= max_block; block += 128) {
      if (launch_dslash(prec, recon, nr, mode, prec, a, block, st) != 0) continue;
      cudaEventRecord(e0, st);
      for (int k = 0; k < reps; ++k) launch_dslash(prec, recon, nr, mode, prec, a, block, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ctx->launches += reps + 1;
      if (cudaGetLastError() == cudaSuccess && ms < best) {
        best = ms;
        best_c.block = block;
        best_c.nr = nr;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(in);
  cudaFree(out);
  cudaFree(aux);
  t->cache[key] = best_c;
  tuner_save(t);
  return best_c;
}

}  // namespace sq
