// Serving loop: many host client threads submit photon bunches; one scheduler
// thread admits them under a fixed budget and runs them in continuous batches.
//
// Paper Sec. 4: the propagation clients queue photon-emitting steps and send
// them, in blocks, to a photon server that aggregates steps from many events
// and clients to keep the GPU busy; several client instances share one server
// and one memory budget.  Here:
//   * pp_submit copies a bunch's sources and queues it (thread-safe);
//   * the scheduler forms a batch from queued bunches, in arrival order, as
//     soon as a batch slot is free and the admission budget allows, so bunches
//     that arrive while others run join the next batch (continuous batching);
//   * each slot owns its device buffers, pinned staging and stream; with
//     several slots in flight, one batch's kernels start while the previous
//     batch's are still finishing;
//   * completion is signalled by a host function queued on the slot's stream
//     (it only posts the slot to the scheduler; no CUDA call inside);
//   * pp_collect waits (bounded) for one bunch's result.
// Results depend only on (seed, event id, sources): a bunch's result is the
// same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pp.h"
#include "pp_internal.h"
#include "pp_nvtx.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket = 0, event_id = 0, n_photons = 0, cost = 0;
  std::vector<pp_source> src;
  Clock::time_point t_submit, t_done;
  int status = 1;  // 1 pending, 0 done, < 0 error
  std::vector<uint64_t> hits;
  uint64_t counts[4] = {0, 0, 0, 0};
};

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  // device
  pp_source* d_src = nullptr;
  int64_t* d_begin = nullptr;
  uint64_t* d_ids = nullptr;
  uint64_t* d_hits = nullptr;
  uint64_t* d_counts = nullptr;
  uint64_t* d_off = nullptr;
  uint32_t* d_chunk = nullptr;
  ppk::SrcAux* d_aux = nullptr;
  uint64_t* d_bsum = nullptr;
  uint64_t* d_meta = nullptr;
  unsigned long long* d_work = nullptr;
  int* d_err = nullptr;
  // pinned host
  pp_source* h_src = nullptr;
  int64_t* h_begin = nullptr;
  uint64_t* h_ids = nullptr;
  uint64_t* h_hits = nullptr;
  uint64_t* h_counts = nullptr;
  int* h_err = nullptr;
  std::vector<Request*> reqs;
  uint64_t cost = 0;
};

}  // namespace

struct pp_server {
  pp_ctx* ctx = nullptr;
  ppk::LaunchView view{};
  pp_server_config cfg{};
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> by_ticket;
  std::deque<int> completed;
  uint64_t next_ticket = 1, in_flight_cost = 0, queued_cost = 0;
  bool stop = false;
  std::thread sched;
  std::string last_error = "no error";
  // statistics
  std::vector<double> latency_ms;
  uint64_t done_requests = 0, done_photons = 0, batches = 0, batch_requests = 0;
  uint64_t peak_cost = 0;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;
};

namespace {

struct HostFnArg {
  pp_server* s;
  int slot;
};

void CUDART_CB on_slot_done(void* p) {
  HostFnArg* a = static_cast<HostFnArg*>(p);
  {
    std::lock_guard<std::mutex> lk(a->s->mu);
    a->s->completed.push_back(a->slot);
  }
  a->s->cv_sched.notify_all();
  delete a;
}

uint64_t request_cost(const pp_server* s, uint64_t n_photons, int64_t n_src) {
  return n_photons * s->cfg.photon_state_bytes + (uint64_t)n_src * 68ull +
         (uint64_t)s->view.geom.n_dom * 8ull + 64ull;
}

bool source_ok(const pp_source& s) {
  return std::isfinite(s.x) && std::isfinite(s.y) && std::isfinite(s.z) && std::isfinite(s.dx) &&
         std::isfinite(s.dy) && std::isfinite(s.dz) && std::isfinite(s.length) && s.length >= 0.f &&
         (s.dx != 0.f || s.dy != 0.f || s.dz != 0.f) && s.type <= PP_SRC_CASCADE;
}

void free_slot(Slot& sl) {
  cudaFree(sl.d_src);
  cudaFree(sl.d_begin);
  cudaFree(sl.d_ids);
  cudaFree(sl.d_hits);
  cudaFree(sl.d_counts);
  cudaFree(sl.d_off);
  cudaFree(sl.d_chunk);
  cudaFree(sl.d_aux);
  cudaFree(sl.d_bsum);
  cudaFree(sl.d_meta);
  cudaFree(sl.d_work);
  cudaFree(sl.d_err);
  cudaFreeHost(sl.h_src);
  cudaFreeHost(sl.h_begin);
  cudaFreeHost(sl.h_ids);
  cudaFreeHost(sl.h_hits);
  cudaFreeHost(sl.h_counts);
  cudaFreeHost(sl.h_err);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  sl = Slot();
}

cudaError_t alloc_slot(Slot& sl, int64_t max_src, int max_req, int n_dom) {
  const int64_t nb = (max_src + ppk::kScanTile - 1) / ppk::kScanTile;
  const size_t hits = sizeof(uint64_t) * (size_t)max_req * std::max(n_dom, 1);
  cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
#define PP_SLOT(x) \
  if (e == cudaSuccess) e = (x)
  PP_SLOT(cudaMalloc(&sl.d_src, sizeof(pp_source) * max_src));
  PP_SLOT(cudaMalloc(&sl.d_begin, sizeof(int64_t) * (max_req + 1)));
  PP_SLOT(cudaMalloc(&sl.d_ids, sizeof(uint64_t) * max_req));
  PP_SLOT(cudaMalloc(&sl.d_hits, hits));
  PP_SLOT(cudaMalloc(&sl.d_counts, sizeof(uint64_t) * 4 * max_req));
  PP_SLOT(cudaMalloc(&sl.d_off, sizeof(uint64_t) * (max_src + 1)));
  PP_SLOT(cudaMalloc(&sl.d_chunk, sizeof(uint32_t) * (max_src + 2)));
  PP_SLOT(cudaMalloc(&sl.d_aux, sizeof(ppk::SrcAux) * max_src));
  PP_SLOT(cudaMalloc(&sl.d_bsum, sizeof(uint64_t) * std::max<int64_t>(nb, 1)));
  PP_SLOT(cudaMalloc(&sl.d_meta, 256));
  PP_SLOT(cudaMalloc(&sl.d_work, 256));
  PP_SLOT(cudaMalloc(&sl.d_err, 256));
  PP_SLOT(cudaMallocHost(&sl.h_src, sizeof(pp_source) * max_src));
  PP_SLOT(cudaMallocHost(&sl.h_begin, sizeof(int64_t) * (max_req + 1)));
  PP_SLOT(cudaMallocHost(&sl.h_ids, sizeof(uint64_t) * max_req));
  PP_SLOT(cudaMallocHost(&sl.h_hits, hits));
  PP_SLOT(cudaMallocHost(&sl.h_counts, sizeof(uint64_t) * 4 * max_req));
  PP_SLOT(cudaMallocHost(&sl.h_err, sizeof(int)));
#undef PP_SLOT
  if (e == cudaSuccess) e = cudaMemset(sl.d_err, 0, 256);
  return e;
}

// Stages a formed batch into the slot and enqueues copies, kernels and the
// completion host function on its stream.  Runs without the server lock (the
// slot and its requests belong to this thread until completion).
cudaError_t launch_slot(pp_server* s, int si) {
  Slot& sl = s->slots[si];
  const int n = (int)sl.reqs.size();
  int64_t n_src = 0;
  sl.h_begin[0] = 0;
  for (int i = 0; i < n; ++i) {
    Request* r = sl.reqs[i];
    std::memcpy(sl.h_src + n_src, r->src.data(), sizeof(pp_source) * r->src.size());
    n_src += (int64_t)r->src.size();
    sl.h_begin[i + 1] = n_src;
    sl.h_ids[i] = r->event_id;
  }
  const int n_dom = s->view.geom.n_dom;
  cudaStream_t st = sl.stream;
  cudaError_t e = cudaMemsetAsync(sl.d_err, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_src, sl.h_src, sizeof(pp_source) * n_src, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_begin, sl.h_begin, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_ids, sl.h_ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_dom)
    e = cudaMemsetAsync(sl.d_hits, 0, sizeof(uint64_t) * (size_t)n * n_dom, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_counts, 0, sizeof(uint64_t) * 4 * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_work, 0, sizeof(uint64_t), st);
  if (e == cudaSuccess && n_src > 0) {
    ppk::ExpandBufs b;
    b.off = sl.d_off;
    b.chunk_src = sl.d_chunk;
    b.aux = sl.d_aux;
    b.bsum = sl.d_bsum;
    b.meta = sl.d_meta;
    e = ppk::launch_expand(sl.d_src, n_src, sl.d_begin, sl.d_ids, n, b, st);
    if (e == cudaSuccess) {
      ppk::WorkDev w{};
      w.src = sl.d_src;
      w.off = sl.d_off;
      w.chunk_src = sl.d_chunk;
      w.aux = sl.d_aux;
      w.meta = sl.d_meta;
      w.work = sl.d_work;
      w.hits = reinterpret_cast<unsigned long long*>(sl.d_hits);
      w.counts = reinterpret_cast<unsigned long long*>(sl.d_counts);
      w.err = sl.d_err;
      w.stats = nullptr;
      w.n_src = (int)n_src;
      w.single_event_lo = 0;
      w.g_begin = 0;
      w.g_end = ~0ull;
      ppk::NvtxRange range("pp.server_batch");
      e = ppk::launch_propagate(true, s->view.ice, s->view.geom, w, s->view.run,
                                s->view.block_threads, s->view.grid_blocks, 0, s->view.smem, st,
                                s->view.variant);
    }
  }
  if (e == cudaSuccess && n_dom)
    e = cudaMemcpyAsync(sl.h_hits, sl.d_hits, sizeof(uint64_t) * (size_t)n * n_dom,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.h_counts, sl.d_counts, sizeof(uint64_t) * 4 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.h_err, sl.d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_slot_done, new HostFnArg{s, si});
  return e;
}

// Results of a completed slot into its requests (server lock held).
void finalize_slot(pp_server* s, int si) {
  Slot& sl = s->slots[si];
  const int n_dom = s->view.geom.n_dom;
  const int err = *sl.h_err;
  const Clock::time_point now = Clock::now();
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    Request* r = sl.reqs[i];
    r->hits.assign(sl.h_hits + i * n_dom, sl.h_hits + (i + 1) * n_dom);
    std::memcpy(r->counts, sl.h_counts + 4 * i, sizeof(r->counts));
    r->status = err ? PP_EDEVICE : PP_OK;
    r->t_done = now;
    s->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
    s->done_requests += 1;
    s->done_photons += r->n_photons;
    r->src.clear();
    r->src.shrink_to_fit();
  }
  s->t_last_done = now;
  s->in_flight_cost -= sl.cost;
  sl.cost = 0;
  sl.reqs.clear();
  sl.busy = false;
}

void fail_slot(pp_server* s, int si, int code) {
  Slot& sl = s->slots[si];
  for (Request* r : sl.reqs) {
    r->status = code;
    r->t_done = Clock::now();
  }
  s->in_flight_cost -= sl.cost;
  sl.cost = 0;
  sl.reqs.clear();
  sl.busy = false;
}

void scheduler(pp_server* s) {
  cudaSetDevice(s->view.device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    auto can_launch = [&]() {
      if (s->pending.empty()) return false;
      for (const Slot& sl : s->slots)
        if (!sl.busy) return s->in_flight_cost + s->pending.front()->cost <= s->cfg.budget_bytes;
      return false;
    };
    auto drained = [&]() {
      if (!s->stop || !s->pending.empty()) return false;
      for (const Slot& sl : s->slots)
        if (sl.busy) return false;
      return true;
    };
    s->cv_sched.wait(lk, [&]() { return !s->completed.empty() || can_launch() || drained(); });
    bool any_done = false;
    while (!s->completed.empty()) {
      const int si = s->completed.front();
      s->completed.pop_front();
      finalize_slot(s, si);
      any_done = true;
    }
    if (any_done) s->cv_done.notify_all();
    if (drained()) break;
    // launch into every free slot while queued work fits the budget
    for (int si = 0; si < (int)s->slots.size(); ++si) {
      Slot& sl = s->slots[si];
      if (sl.busy || s->pending.empty()) continue;
      int64_t n_src = 0;
      while (!s->pending.empty()) {
        Request* r = s->pending.front();
        if ((int)sl.reqs.size() >= s->cfg.max_batch_requests) break;
        if (n_src + (int64_t)r->src.size() > s->cfg.max_batch_sources) break;
        if (s->in_flight_cost + sl.cost + r->cost > s->cfg.budget_bytes) break;
        s->pending.pop_front();
        s->queued_cost -= r->cost;
        sl.reqs.push_back(r);
        sl.cost += r->cost;
        n_src += (int64_t)r->src.size();
      }
      if (sl.reqs.empty()) break;  // the budget is full: wait for a completion
      sl.busy = true;
      s->in_flight_cost += sl.cost;
      s->peak_cost = std::max(s->peak_cost, s->in_flight_cost);
      s->batches += 1;
      s->batch_requests += sl.reqs.size();
      lk.unlock();
      const cudaError_t e = launch_slot(s, si);
      lk.lock();
      if (e != cudaSuccess) {
        s->last_error = std::string("batch launch: ") + cudaGetErrorString(e);
        fail_slot(s, si, PP_ECUDA);
        s->cv_done.notify_all();
      }
    }
  }
  // fail anything left (only reachable on stop with nothing pending)
  s->cv_done.notify_all();
}

}  // namespace

extern "C" {

int pp_server_config_default(pp_server_config* cfg) {
  if (!cfg) return PP_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->budget_bytes = 8ull << 30;
  cfg->photon_state_bytes = 32;
  cfg->slots = 3;
  cfg->max_batch_requests = 512;
  cfg->max_batch_sources = 1 << 20;
  return PP_OK;
}

int pp_server_create(pp_ctx* ctx, const pp_server_config* cfg, pp_server** out) {
  if (!ctx || !cfg || !out) return PP_EINVAL;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch_requests < 1 ||
      cfg->max_batch_sources < 1 || cfg->max_batch_sources > ppk::kMaxSources ||
      cfg->budget_bytes == 0)
    return PP_EINVAL;
  pp_server* s = new pp_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  const int rc = ppk::with_launch_view(ctx, [&](const ppk::LaunchView& v) {
    s->view = v;
    ppk::attach_server(ctx, +1);  // the context refuses new tables while attached
    return PP_OK;
  });
  if (rc) {
    delete s;
    return rc;
  }
  ppk::DeviceScope dev_scope(s->view.device);
  s->slots.resize(cfg->slots);
  for (Slot& sl : s->slots) {
    if (alloc_slot(sl, cfg->max_batch_sources, cfg->max_batch_requests, s->view.geom.n_dom) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      for (Slot& x : s->slots) free_slot(x);
      ppk::attach_server(ctx, -1);
      delete s;
      return PP_ENOMEM;
    }
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return PP_OK;
}

int pp_server_destroy(pp_server* s) {
  if (!s) return PP_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->sched.joinable()) s->sched.join();
  ppk::DeviceScope dev_scope(s->view.device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    free_slot(sl);
  }
  for (auto& kv : s->by_ticket) delete kv.second;
  ppk::attach_server(s->ctx, -1);
  delete s;
  return PP_OK;
}

const char* pp_server_last_error(const pp_server* s) {
  return s ? s->last_error.c_str() : "null server";
}

int pp_submit(pp_server* s, uint64_t event_id, const pp_source* src, int64_t n_src,
              uint64_t* ticket_out) {
  if (!s || !ticket_out || n_src < 0 || (n_src > 0 && !src)) return PP_EINVAL;
  if (n_src > s->cfg.max_batch_sources) return PP_EINVAL;
  uint64_t n_photons = 0;
  for (int64_t i = 0; i < n_src; ++i) {
    if (!source_ok(src[i])) return PP_EINVAL;
    n_photons += src[i].n_photons;
  }
  const uint64_t cost = request_cost(s, n_photons, n_src);
  if (cost > s->cfg.budget_bytes) return PP_EBUDGET;
  Request* r = new Request();
  r->event_id = event_id;
  r->n_photons = n_photons;
  r->cost = cost;
  r->src.assign(src, src + n_src);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return PP_EINVAL;
    }
    r->ticket = s->next_ticket++;
    s->by_ticket[r->ticket] = r;
    s->pending.push_back(r);
    s->queued_cost += cost;
    if (!s->any_submit) {
      s->any_submit = true;
      s->t_first_submit = r->t_submit;
    }
    *ticket_out = r->ticket;
  }
  s->cv_sched.notify_all();
  return PP_OK;
}

int pp_collect(pp_server* s, uint64_t ticket, uint64_t* hits, uint64_t* counts,
               int32_t timeout_ms) {
  if (!s) return PP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return PP_EINVAL;
  Request* r = it->second;
  auto ready = [&]() { return r->status != 1; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return PP_ETIMEDOUT;
  }
  const int st = r->status;
  if (st == PP_OK) {
    if (hits && !r->hits.empty()) std::memcpy(hits, r->hits.data(), sizeof(uint64_t) * r->hits.size());
    if (counts) std::memcpy(counts, r->counts, sizeof(r->counts));
  }
  s->by_ticket.erase(it);
  delete r;
  return st;
}

int pp_server_stats(pp_server* s, double* out8) {
  if (!s || !out8) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->latency_ms;
  std::sort(v.begin(), v.end());
  auto q = [&](double p) {
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
    return v[i];
  };
  const double span =
      s->any_submit ? std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count() : 0.0;
  out8[0] = (double)s->done_requests;
  out8[1] = (double)s->done_photons;
  out8[2] = q(0.50);
  out8[3] = q(0.99);
  out8[4] = span > 0 ? (double)s->done_photons / span : 0.0;
  out8[5] = s->batches ? (double)s->batch_requests / (double)s->batches : 0.0;
  out8[6] = (double)s->batches;
  out8[7] = (double)s->peak_cost;
  return PP_OK;
}

}  // extern "C"
