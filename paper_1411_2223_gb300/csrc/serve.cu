// Continuous-batching serving engine for CG solves.
//
// A scheduler thread owns one batch per gauge field: a batched mixed-precision
// CG workspace with S slots on its own CUDA stream.  Batches of different
// gauge fields run concurrently on the device.  Each batch advances in graph
// blocks of k iterations (k a multiple of the reliable-update period).
// Between blocks the scheduler
//   * retires the slots whose system finished (solution copied to the
//     request, latency recorded, pollers woken),
//   * admits queued requests into free slots: source uploaded and packed, the
//     slot put in SLOT_INIT and started by the init kernel while the other
//     slots keep their state -- a request joins a running batch,
//   * launches the next block if any slot is live.
// A batch's device memory is taken from the context's HBM budget when its
// first request arrives; if the budget refuses, idle batches of other gauge
// fields are released and the requests wait (admission by HBM footprint).
// Because admissions happen only at block boundaries, which are checkpoint
// boundaries, a system follows exactly the same arithmetic alone or in a
// mixed batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "serve.h"
#include "sq_host.h"

namespace sq {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int gid = 0;
  double mass = 0, tol = 0;
  std::vector<double> src;  // canonical host copy
  std::vector<double> x;
  sq_cg_stats stats{};
  int status = SQ_PENDING;
  bool done = false, cancelled = false;
  Clock::time_point t_submit, t_done;
};

struct Batch {
  int gid = 0;
  GaugeField *gf = nullptr;
  CGWork *w = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<std::shared_ptr<Request>> slot;
  std::deque<std::shared_ptr<Request>> pending;
  double *pin = nullptr;     // pinned staging, S canonical vectors
  double *canon = nullptr;   // device staging, S canonical vectors
  size_t vec = 0;            // doubles per canonical vector
  bool inflight = false;
  bool drop = false;         // release requested (gauge_free)

  bool busy() const {
    if (!pending.empty()) return true;
    for (auto &r : slot)
      if (r) return true;
    return false;
  }
  void release_device(sq_ctx *ctx) {
    if (st) cudaStreamSynchronize(st);
    delete w;
    w = nullptr;
    if (canon) ctx->release(canon, vec * sizeof(double) * slot.size());
    canon = nullptr;
    if (pin) cudaFreeHost(pin);
    pin = nullptr;
  }
};

}  // namespace

struct ServeEngine {
  sq_ctx *ctx = nullptr;
  int slots = 8, block_iters = 8;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> incoming;
  std::map<int, std::unique_ptr<Batch>> batches;  // scheduler thread only (+ under mu)
  std::thread th;
  bool stop = false;
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0, rejected = 0;
  std::vector<double> lat_ms;
  Clock::time_point first_submit, last_done;
  bool have_first = false;
  std::atomic<int> running_slots{0};

  void loop();
  bool step_batch(Batch &b);
};

static void finish_request(ServeEngine *e, Batch &b, int s) {
  auto &req = b.slot[s];
  const SlotState &ss = b.w->slots_h[s];
  std::memcpy(req->x.data(), b.pin + (size_t)s * b.vec, b.vec * sizeof(double));
  auto now = Clock::now();
  double secs = std::chrono::duration<double>(now - req->t_submit).count();
  fill_stats(ss, secs, b.gf->g.vh, &req->stats);
  fill_launch_stats(b.w, &req->stats);
  {
    std::lock_guard<std::mutex> lk(e->mu);
    req->status = req->stats.status;
    req->t_done = now;
    req->done = true;
    if (!req->cancelled) {
      e->completed++;
      e->lat_ms.push_back(secs * 1e3);
      e->last_done = now;
    }
    b.w->slots_h[s].status = SLOT_IDLE;
    req.reset();
  }
  e->cv_done.notify_all();
}

// One scheduling step of a batch; returns true if it launched GPU work.
bool ServeEngine::step_batch(Batch &b) {
  if (b.inflight) {
    cudaError_t q = cudaEventQuery(b.ev);
    if (q == cudaErrorNotReady) return false;
    b.inflight = false;
  }
  if (!b.w) {
    if (b.pending.empty()) return false;
    CGWork *w = nullptr;
    int rc = cg_work_create(ctx, b.gf, PREC_F32, 18, slots, &w);
    if (rc == SQ_ERR_OOM) {  // free idle batches of other fields, then retry
      for (auto &kv : batches)
        if (kv.second.get() != &b && kv.second->w && !kv.second->busy() && !kv.second->inflight)
          kv.second->release_device(ctx);
      rc = cg_work_create(ctx, b.gf, PREC_F32, 18, slots, &w);
    }
    if (rc != SQ_OK) return false;  // stays queued: admitted when memory frees up
    b.vec = (size_t)6 * b.gf->g.vh;
    if (ctx->alloc(b.vec * sizeof(double) * slots, (void **)&b.canon) != SQ_OK ||
        cudaMallocHost((void **)&b.pin, b.vec * sizeof(double) * slots) != cudaSuccess) {
      delete w;
      if (b.canon) ctx->release(b.canon, b.vec * sizeof(double) * slots);
      b.canon = nullptr;
      return false;
    }
    w->cfg_norm = tuned_dslash(ctx, *b.gf, PREC_F32, 18, slots, MODE_NORM, b.st);
    w->cfg_update = tuned_dslash(ctx, *b.gf, PREC_F32, 18, slots, MODE_UPDATE, b.st);
    w->cfg_ru_plain = tuned_dslash(ctx, *b.gf, PREC_F64, 18, slots, MODE_PLAIN, b.st);
    w->cfg_ru_resid = w->cfg_ru_plain;
    b.w = w;
  }
  CGWork *w = b.w;
  // retire finished slots and drop cancelled ones
  std::vector<int> done;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int s = 0; s < slots; ++s) {
      if (!b.slot[s]) continue;
      if (b.slot[s]->cancelled) {
        w->slots_h[s].status = SLOT_IDLE;
        b.slot[s].reset();
        continue;
      }
      if (!cg_slot_live(w->slots_h[s].status)) done.push_back(s);
    }
  }
  const Geom &g = b.gf->g;
  const size_t vb = b.vec * sizeof(double);
  for (int s : done) {
    launch_unpack(PREC_F64, g, w->x64 + (size_t)s * w->f64_fb, 0, b.canon + (size_t)s * b.vec, 0,
                  1, b.st);
    cudaMemcpyAsync(b.pin + (size_t)s * b.vec, b.canon + (size_t)s * b.vec, vb,
                    cudaMemcpyDeviceToHost, b.st);
    ctx->launches++;
  }
  if (!done.empty()) {
    cudaStreamSynchronize(b.st);
    for (int s : done) finish_request(this, b, s);
  }
  // admit queued requests into free slots
  bool admitted = false;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int s = 0; s < slots && !b.pending.empty(); ++s) {
      if (b.slot[s]) continue;
      auto req = b.pending.front();
      b.pending.pop_front();
      if (req->cancelled) {
        --s;
        continue;
      }
      b.slot[s] = req;
      std::memcpy(b.pin + (size_t)s * b.vec, req->src.data(), vb);
      cudaMemcpyAsync(b.canon + (size_t)s * b.vec, b.pin + (size_t)s * b.vec, vb,
                      cudaMemcpyHostToDevice, b.st);
      launch_pack(PREC_F64, g, b.canon + (size_t)s * b.vec, 0, w->b64 + (size_t)s * w->f64_fb,
                  0, 1, b.st);
      ctx->launches++;
      cg_slot_setup(w, s, req->mass, req->tol, 0.01, 100000);
      admitted = true;
    }
  }
  if (admitted) {
    cg_slots_upload(w, b.st);
    cg_enqueue_init(w, 0, b.st);
  }
  bool live = false;
  int nlive = 0;
  for (int s = 0; s < slots; ++s)
    if (b.slot[s] && cg_slot_live(w->slots_h[s].status)) {
      live = true;
      ++nlive;
    }
  if (admitted) live = true;
  if (!live) return false;
  if (cg_enqueue_block(w, block_iters, true, b.st) != SQ_OK) {
    // a launch failure ends the batch's systems with an error
    {
      std::lock_guard<std::mutex> lk(mu);
      for (int s = 0; s < slots; ++s)
        if (b.slot[s]) {
          b.slot[s]->status = SQ_ERR_CUDA;
          b.slot[s]->done = true;
          b.slot[s].reset();
        }
    }
    cv_done.notify_all();
    return false;
  }
  cg_slots_download(w, b.st);
  cudaEventRecord(b.ev, b.st);
  b.inflight = true;
  return true;
}

void ServeEngine::loop() {
  cudaSetDevice(ctx->device);
  while (true) {
    {
      std::unique_lock<std::mutex> lk(mu);
      if (stop) break;
      while (!incoming.empty()) {
        auto r = incoming.front();
        incoming.pop_front();
        auto &bp = batches[r->gid];
        if (!bp) {
          bp.reset(new Batch());
          bp->gid = r->gid;
          bp->gf = ctx->gauge(r->gid);
          bp->slot.resize(slots);
          cudaStreamCreateWithFlags(&bp->st, cudaStreamNonBlocking);
          cudaEventCreateWithFlags(&bp->ev, cudaEventDisableTiming);
        }
        bp->pending.push_back(r);
      }
    }
    bool any_inflight = false, any_pending = false;
    int live = 0;
    for (auto &kv : batches) {
      Batch &b = *kv.second;
      step_batch(b);
      std::lock_guard<std::mutex> lk(mu);
      any_inflight |= b.inflight;
      any_pending |= !b.pending.empty();
      for (auto &r : b.slot) live += r ? 1 : 0;
    }
    running_slots = live;
    {  // release batches whose gauge field is being freed
      std::lock_guard<std::mutex> lk(mu);
      for (auto it = batches.begin(); it != batches.end();) {
        Batch &b = *it->second;
        if (b.drop && !b.busy() && !b.inflight) {
          b.release_device(ctx);
          if (b.ev) cudaEventDestroy(b.ev);
          if (b.st) cudaStreamDestroy(b.st);
          it = batches.erase(it);
          cv_done.notify_all();
        } else {
          ++it;
        }
      }
    }
    std::unique_lock<std::mutex> lk(mu);
    if (stop) break;
    if (!any_inflight && incoming.empty()) {
      // nothing on the device: sleep until a submission (or a pending retry)
      cv_work.wait_for(lk, std::chrono::milliseconds(any_pending ? 1 : 50));
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  for (auto &kv : batches) {
    kv.second->release_device(ctx);
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    if (kv.second->st) cudaStreamDestroy(kv.second->st);
  }
  batches.clear();
}

static ServeEngine *engine(sq_ctx *ctx) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->serve) {
    ServeEngine *e = new ServeEngine();
    e->ctx = ctx;
    ctx->serve = e;
  }
  return ctx->serve;
}

static void ensure_thread(ServeEngine *e) {
  if (!e->th.joinable()) e->th = std::thread([e] { e->loop(); });
}

void serve_shutdown(ServeEngine *e) {
  if (!e) return;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->stop = true;
  }
  e->cv_work.notify_all();
  if (e->th.joinable()) e->th.join();
  delete e;
}

bool serve_uses_gauge(ServeEngine *e, int gauge_id) {
  std::unique_lock<std::mutex> lk(e->mu);
  for (auto &r : e->incoming)
    if (r->gid == gauge_id) return true;
  auto it = e->batches.find(gauge_id);
  if (it == e->batches.end()) return false;
  if (it->second->busy()) return true;
  if (!e->th.joinable()) return true;
  it->second->drop = true;  // the scheduler releases it between blocks
  e->cv_work.notify_all();
  e->cv_done.wait_for(lk, std::chrono::seconds(30),
                      [&] { return e->batches.find(gauge_id) == e->batches.end(); });
  return e->batches.find(gauge_id) != e->batches.end();
}

}  // namespace sq

using namespace sq;

extern "C" int serve_configure(sq_ctx *ctx, int slots_per_batch, int block_iters) {
  if (!ctx || slots_per_batch < 1 || slots_per_batch > 16 || block_iters < 1) return SQ_ERR_ARG;
  ServeEngine *e = engine(ctx);
  std::lock_guard<std::mutex> lk(e->mu);
  if (!e->batches.empty() || !e->incoming.empty()) return SQ_ERR_BUSY;
  e->slots = slots_per_batch;
  e->block_iters = (block_iters + RU_PERIOD - 1) / RU_PERIOD * RU_PERIOD;
  return SQ_OK;
}

extern "C" int serve_submit(sq_ctx *ctx, int gauge_id, const double *src_even, double mass,
                            double tol, uint64_t *ticket) {
  if (!ctx || !src_even || !ticket) return SQ_ERR_ARG;
  if (!(mass > 0) || !std::isfinite(mass) || !(tol > 0) || !std::isfinite(tol)) return SQ_ERR_ARG;
  GaugeField *gf = ctx->gauge(gauge_id);
  if (!gf) return SQ_ERR_NOTFOUND;
  if (!gf->has(PREC_F32, 18) || !gf->has(PREC_F64, 18)) return SQ_ERR_UNSUPPORTED;
  const size_t n = (size_t)6 * gf->g.vh;
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(src_even[k])) return SQ_ERR_NONFINITE;
  auto r = std::make_shared<Request>();
  r->gid = gauge_id;
  r->mass = mass;
  r->tol = tol;
  r->src.assign(src_even, src_even + n);
  r->x.assign(n, 0.0);
  r->t_submit = Clock::now();
  ServeEngine *e = engine(ctx);
  {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->stop) return SQ_ERR_BUSY;
    r->ticket = e->next_ticket++;
    e->reqs[r->ticket] = r;
    e->incoming.push_back(r);
    e->submitted++;
    if (!e->have_first) {
      e->first_submit = r->t_submit;
      e->have_first = true;
    }
    ensure_thread(e);
  }
  e->cv_work.notify_all();
  *ticket = r->ticket;
  return SQ_OK;
}

extern "C" int serve_poll(sq_ctx *ctx, uint64_t ticket, double *x_even, sq_cg_stats *stats,
                          int timeout_us) {
  if (!ctx) return SQ_ERR_ARG;
  ServeEngine *e = engine(ctx);
  std::unique_lock<std::mutex> lk(e->mu);
  auto it = e->reqs.find(ticket);
  if (it == e->reqs.end()) return SQ_ERR_NOTFOUND;
  std::shared_ptr<Request> r = it->second;
  if (!r->done && timeout_us != 0) {
    auto pred = [&] { return r->done; };
    if (timeout_us < 0) e->cv_done.wait(lk, pred);
    else e->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
  }
  if (!r->done) return SQ_PENDING;
  if (x_even) std::memcpy(x_even, r->x.data(), r->x.size() * sizeof(double));
  if (stats) *stats = r->stats;
  e->reqs.erase(ticket);
  return r->status;
}

extern "C" int serve_cancel(sq_ctx *ctx, uint64_t ticket) {
  if (!ctx) return SQ_ERR_ARG;
  ServeEngine *e = engine(ctx);
  std::lock_guard<std::mutex> lk(e->mu);
  auto it = e->reqs.find(ticket);
  if (it == e->reqs.end()) return SQ_ERR_NOTFOUND;
  it->second->cancelled = true;  // the scheduler frees its slot between blocks
  e->reqs.erase(it);
  return SQ_OK;
}

extern "C" int serve_stats(sq_ctx *ctx, sq_serve_stats *st, int reset) {
  if (!ctx || !st) return SQ_ERR_ARG;
  ServeEngine *e = engine(ctx);
  std::lock_guard<std::mutex> lk(e->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = e->submitted;
  st->completed = e->completed;
  st->rejected = e->rejected;
  st->queued = (int)e->incoming.size();
  for (auto &kv : e->batches) st->queued += (int)kv.second->pending.size();
  st->running = e->running_slots.load();
  std::vector<double> v = e->lat_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      double pos = q * (v.size() - 1);
      size_t lo = (size_t)pos;
      size_t hi = std::min(lo + 1, v.size() - 1);
      return v[lo] + (pos - lo) * (v[hi] - v[lo]);
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_ms = sum / v.size();
    double span = std::chrono::duration<double>(e->last_done - e->first_submit).count();
    st->solves_per_s = span > 0 ? e->completed / span : 0;
  }
  {
    std::lock_guard<std::mutex> l2(ctx->mu);
    st->hbm_in_use = ctx->in_use;
    st->hbm_budget = ctx->budget;
  }
  if (reset) {
    e->lat_ms.clear();
    e->completed = e->submitted = e->rejected = 0;
    e->have_first = false;
  }
  return SQ_OK;
}
