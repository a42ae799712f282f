// Serving loop: many host client threads submit photon bunches; the bunches
// are admitted into a request ring in device memory, and a persistent serving
// kernel pulls photons from the ring while requests keep arriving.
//
// Paper Sec. 4: the propagation clients queue photon-emitting steps and send
// them, in blocks, to a photon server that aggregates steps from many events
// and clients to keep the GPU busy; several client instances share one server
// and one memory budget.  Here:
//   * pp_submit (any client thread) checks a bunch, computes its photon prefix
//     and photon-chunk table on the host, and queues it for admission;
//   * the scheduler thread admits queued bunches in arrival order while a
//     ring slot, arena space and the budget allow: it copies the sources,
//     prefix and chunk table into device arenas, clears the slot's outputs,
//     writes the ring entry and finally the ring's tail (the doorbell), all as
//     copies on one stream, so the device sees a request only once its data is
//     in place;
//   * the serving kernel (k_serve) claims up to 32 photons at a time from the
//     oldest request with unclaimed photons (an atomic add to its ring
//     slot's claim word), runs them with the batched
//     kernel's per-warp photon reserve, tallies them into the request's
//     outputs and raises the request's host-mapped done flag when its last
//     photon is tallied.  Requests that arrive while it runs are taken by the
//     running kernel (continuous batching on the device); it leaves when idle,
//     or after a time limit, and the scheduler relaunches it while published
//     requests are unfinished;
//   * the scheduler copies a finished request's outputs back and wakes its
//     collector.
// Admission charges the device bytes a request actually occupies while
// admitted (its sources, prefix and chunk table in the arenas, its output
// slot and ring entry): photon state lives in registers and in shared memory,
// never in device memory.  Results depend only on (seed, event id, sources):
// a bunch's result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
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

constexpr int kQueued = 1, kPublished = 2, kCopying = 3;

struct Request {
  uint64_t ticket = 0, event_id = 0, n_photons = 0, bytes = 0;
  std::vector<pp_source> src;
  std::vector<uint64_t> off;     // photon prefix over the sources (n_src + 1)
  std::vector<uint32_t> chunk;   // photon-chunk -> first source (n_chunks + 1)
  uint32_t chunk_log2 = 0;
  Clock::time_point t_submit, t_done;
  int status = kQueued;          // kQueued, kPublished, kCopying, 0 done, < 0 error
  uint64_t seq = 0;
  int slot = -1;
  uint64_t src_at = 0, off_at = 0, chunk_at = 0;
  std::vector<uint64_t> hits;
  uint64_t counts[4] = {0, 0, 0, 0};
};

// First-fit allocator of ranges [0, cap) with coalescing of freed ranges.
class RangeAlloc {
 public:
  void reset(uint64_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool take(uint64_t n, uint64_t* at) {
    if (n == 0) {
      *at = 0;
      return true;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *at = it->first;
        const uint64_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void give(uint64_t at, uint64_t n) {
    if (n == 0) return;
    auto next = free_.lower_bound(at);
    if (next != free_.end() && at + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == at) {
        prev->second += n;
        return;
      }
    }
    free_[at] = n;
  }

 private:
  std::map<uint64_t, uint64_t> free_;
};

}  // namespace

struct pp_server {
  pp_ctx* ctx = nullptr;
  ppk::LaunchView view{};
  pp_server_config cfg{};
  int cap = 0;                 // ring slots (a power of two)
  int grid = 0;                // serving kernel blocks
  size_t smem = 0;
  // device
  ppk::ServeReq* d_req = nullptr;
  unsigned long long* d_tail = nullptr;
  unsigned long long* d_head = nullptr;
  int* d_may_leave = nullptr;           // 1: the kernel's idle warps may close the launch
  int* d_closing = nullptr;             // the launch is closing (cleared before each launch)
  pp_source* d_src = nullptr;
  uint64_t* d_off = nullptr;
  uint32_t* d_chunk = nullptr;
  uint64_t* d_hits = nullptr;
  uint64_t* d_counts = nullptr;
  int* d_err = nullptr;
  uint64_t device_bytes = 0;
  // pinned host: staging mirrors of the arenas and the ring, result landing
  // areas, the host-mapped done flags
  pp_source* h_src = nullptr;
  uint64_t* h_off = nullptr;
  uint32_t* h_chunk = nullptr;
  ppk::ServeReq* h_req = nullptr;
  unsigned long long* h_tail = nullptr;  // [cap]: the tail value each publication writes
  unsigned long long* h_arm = nullptr;   // [cap]: the claim word that arms each slot
  uint64_t* h_zero = nullptr;            // n_dom + 4 zeros
  int* h_one = nullptr;                  // a pinned 1 (the may-leave flag's value)
  uint64_t* h_hits = nullptr;
  uint64_t* h_counts = nullptr;
  int* h_err = nullptr;                  // [cap]
  volatile uint32_t* h_flag = nullptr;   // [cap], device-mapped
  uint32_t* d_flag = nullptr;            // its device address
  cudaStream_t s_pub = nullptr, s_down = nullptr, s_kern = nullptr;
  cudaEvent_t kern_done = nullptr;
  std::vector<cudaEvent_t> copied;       // [cap]
  bool kernel_running = false;
  bool may_leave = false;                // the last value written to d_may_leave
  // host state
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> by_slot;         // [cap]: the admitted request in each slot
  std::unordered_map<uint64_t, Request*> by_ticket;
  RangeAlloc a_src, a_off, a_chunk;
  uint64_t next_ticket = 1, next_seq = 0, admitted_bytes = 0, published = 0;
  bool stop = false, broken = false;
  std::thread sched;
  std::string last_error = "no error";
  // statistics
  std::vector<double> latency_ms;
  uint64_t done_requests = 0, done_photons = 0, launches = 0, peak_bytes = 0;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;
};

namespace {

bool source_ok(const pp_source& s) {
  return std::isfinite(s.x) && std::isfinite(s.y) && std::isfinite(s.z) && std::isfinite(s.dx) &&
         std::isfinite(s.dy) && std::isfinite(s.dz) && std::isfinite(s.length) && s.length >= 0.f &&
         (s.dx != 0.f || s.dy != 0.f || s.dz != 0.f) && s.type <= PP_SRC_CASCADE;
}

// a1 for one request, on the host: the exclusive photon prefix over its
// sources and the table of 2^k-photon chunks (k the smallest with at most
// n_src + 1 chunks) -> the last source starting at or before the chunk's
// first photon, as the device expansion builds them for a batch.
void expand_on_host(Request* r) {
  const size_t n = r->src.size();
  r->off.resize(n + 1);
  uint64_t acc = 0;
  for (size_t i = 0; i < n; ++i) {
    r->off[i] = acc;
    acc += r->src[i].n_photons;
  }
  r->off[n] = acc;
  r->n_photons = acc;
  uint32_t k = 0;
  const uint64_t cap = std::max<uint64_t>(n, 1);
  while ((acc >> k) > cap) ++k;
  r->chunk_log2 = k;
  const uint64_t n_chunks = (acc + (1ull << k) - 1) >> k;
  r->chunk.resize(n_chunks + 1);
  size_t s = 0;
  for (uint64_t c = 0; c <= n_chunks; ++c) {
    const uint64_t g = c << k;
    while (s + 1 < n && r->off[s + 1] <= g) ++s;
    r->chunk[c] = (uint32_t)s;
  }
}

// Device bytes a request occupies while admitted: its sources, prefix and
// chunk table in the arenas, its output slot and its ring entry.
uint64_t request_bytes(const pp_server* s, const Request* r) {
  return sizeof(pp_source) * r->src.size() + sizeof(uint64_t) * r->off.size() +
         sizeof(uint32_t) * r->chunk.size() +
         sizeof(uint64_t) * ((uint64_t)s->view.geom.n_dom + 4) + sizeof(ppk::ServeReq);
}

void free_server_memory(pp_server* s) {
  void* dev[] = {s->d_req, s->d_tail, s->d_head, s->d_may_leave, s->d_closing, s->d_src, s->d_off, s->d_chunk,
                 s->d_hits, s->d_counts, s->d_err};
  for (void* p : dev) cudaFree(p);
  void* host[] = {s->h_src, s->h_off, s->h_chunk, s->h_req, s->h_tail, s->h_arm, s->h_zero, s->h_one,
                  s->h_hits, s->h_counts, s->h_err, (void*)s->h_flag};
  for (void* p : host) cudaFreeHost(p);
  for (cudaEvent_t e : s->copied) cudaEventDestroy(e);
  if (s->kern_done) cudaEventDestroy(s->kern_done);
  if (s->s_pub) cudaStreamDestroy(s->s_pub);
  if (s->s_down) cudaStreamDestroy(s->s_down);
  if (s->s_kern) cudaStreamDestroy(s->s_kern);
}

template <class T>
cudaError_t dev_alloc(pp_server* s, T** p, size_t n) {
  const size_t b = sizeof(T) * std::max<size_t>(n, 1);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), b);
  if (e == cudaSuccess) s->device_bytes += b;
  return e;
}

cudaError_t alloc_server_memory(pp_server* s) {
  const size_t S = (size_t)s->cfg.arena_sources, R = (size_t)s->cap;
  const size_t n_dom = (size_t)std::max(s->view.geom.n_dom, 1);
  cudaError_t e = cudaSuccess;
#define PP_A(x) \
  if (e == cudaSuccess) e = (x)
  PP_A(dev_alloc(s, &s->d_req, R));
  PP_A(dev_alloc(s, &s->d_tail, 1));
  PP_A(dev_alloc(s, &s->d_head, 1));
  PP_A(dev_alloc(s, &s->d_may_leave, 1));
  PP_A(dev_alloc(s, &s->d_closing, 1));
  PP_A(dev_alloc(s, &s->d_src, S));
  PP_A(dev_alloc(s, &s->d_off, S + R));
  PP_A(dev_alloc(s, &s->d_chunk, S + 2 * R));
  PP_A(dev_alloc(s, &s->d_hits, R * n_dom));
  PP_A(dev_alloc(s, &s->d_counts, R * 4));
  PP_A(dev_alloc(s, &s->d_err, 1));
  PP_A(cudaMallocHost(&s->h_src, sizeof(pp_source) * std::max<size_t>(S, 1)));
  PP_A(cudaMallocHost(&s->h_off, sizeof(uint64_t) * (S + R)));
  PP_A(cudaMallocHost(&s->h_chunk, sizeof(uint32_t) * (S + 2 * R)));
  PP_A(cudaMallocHost(&s->h_req, sizeof(ppk::ServeReq) * R));
  PP_A(cudaMallocHost(&s->h_tail, sizeof(unsigned long long) * R));
  PP_A(cudaMallocHost(&s->h_arm, sizeof(unsigned long long) * R));
  PP_A(cudaMallocHost(&s->h_zero, sizeof(uint64_t) * (n_dom + 4)));
  PP_A(cudaMallocHost(&s->h_one, sizeof(int)));
  PP_A(cudaMallocHost(&s->h_hits, sizeof(uint64_t) * R * n_dom));
  PP_A(cudaMallocHost(&s->h_counts, sizeof(uint64_t) * R * 4));
  PP_A(cudaMallocHost(&s->h_err, sizeof(int) * R));
  void* flag = nullptr;
  PP_A(cudaHostAlloc(&flag, sizeof(uint32_t) * R, cudaHostAllocMapped));
  if (e == cudaSuccess) {
    s->h_flag = static_cast<volatile uint32_t*>(flag);
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_flag), flag, 0);
  }
  PP_A(cudaStreamCreateWithFlags(&s->s_pub, cudaStreamNonBlocking));
  PP_A(cudaStreamCreateWithFlags(&s->s_down, cudaStreamNonBlocking));
  PP_A(cudaStreamCreateWithFlags(&s->s_kern, cudaStreamNonBlocking));
  PP_A(cudaEventCreateWithFlags(&s->kern_done, cudaEventDisableTiming));
  s->copied.assign(R, nullptr);
  for (size_t i = 0; i < R && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming);
#undef PP_A
  if (e != cudaSuccess) return e;
  std::memset(s->h_zero, 0, sizeof(uint64_t) * (n_dom + 4));
  *s->h_one = 1;
  for (size_t i = 0; i < R; ++i) s->h_flag[i] = 0;
  // the ring starts empty (tail and head 0) with every slot disarmed (a
  // claim word whose request number matches no slot's seq), no error
  ppk::ServeReq* init = s->h_req;
  for (size_t i = 0; i < R; ++i) {
    std::memset(&init[i], 0, sizeof(ppk::ServeReq));
    init[i].claimed = (((1ull << ppk::kServeSeqBits) - 1) << ppk::kServeOffsetBits) |
                      ppk::kServeMaxPhotons;
    init[i].seq = ~0u;
  }
  e = cudaMemcpyAsync(s->d_req, init, sizeof(ppk::ServeReq) * R, cudaMemcpyHostToDevice, s->s_pub);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_tail, 0, sizeof(unsigned long long), s->s_pub);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_head, 0, sizeof(unsigned long long), s->s_pub);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_may_leave, 0, sizeof(int), s->s_pub);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->s_pub);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_pub);
  s->a_src.reset(S);
  s->a_off.reset(S + R);
  s->a_chunk.reset(S + 2 * R);
  return e;
}

// Admits the oldest queued request if a ring slot, arena space and the budget
// allow (server lock held).  Its data go to the device as copies on the
// publication stream, the ring entry and the tail last.  Returns false when
// the request has to wait.
bool admit_front(pp_server* s) {
  Request* r = s->pending.front();
  const int slot = (int)(s->next_seq & (uint64_t)(s->cap - 1));
  if (s->by_slot[slot]) return false;  // the slot's previous request is not collected back yet
  if (s->admitted_bytes + r->bytes > s->cfg.budget_bytes) return false;
  uint64_t a = 0, b = 0, c = 0;
  if (!s->a_src.take(r->src.size(), &a)) return false;
  if (!s->a_off.take(r->off.size(), &b)) {
    s->a_src.give(a, r->src.size());
    return false;
  }
  if (!s->a_chunk.take(r->chunk.size(), &c)) {
    s->a_src.give(a, r->src.size());
    s->a_off.give(b, r->off.size());
    return false;
  }
  s->pending.pop_front();
  r->src_at = a;
  r->off_at = b;
  r->chunk_at = c;
  r->slot = slot;
  r->seq = s->next_seq++;
  s->by_slot[slot] = r;
  s->admitted_bytes += r->bytes;
  s->peak_bytes = std::max(s->peak_bytes, s->admitted_bytes);
  const int n_dom = s->view.geom.n_dom;
  // stage into the pinned mirrors (the ranges are this request's alone)
  std::memcpy(s->h_src + a, r->src.data(), sizeof(pp_source) * r->src.size());
  std::memcpy(s->h_off + b, r->off.data(), sizeof(uint64_t) * r->off.size());
  std::memcpy(s->h_chunk + c, r->chunk.data(), sizeof(uint32_t) * r->chunk.size());
  ppk::ServeReq& q = s->h_req[slot];
  q.claimed = 0;  // not copied: the arming copy below writes it
  q.done = 0;
  q.total = r->n_photons;
  q.src_off = a;
  q.off_off = b;
  q.chunk_off = c;
  q.n_src = (uint32_t)r->src.size();
  q.chunk_log2 = r->chunk_log2;
  q.event_lo = (uint32_t)r->event_id;
  q.seq = (uint32_t)r->seq;
  s->h_arm[slot] = (r->seq & ((1ull << ppk::kServeSeqBits) - 1)) << ppk::kServeOffsetBits;
  s->h_tail[slot] = r->seq + 1;
  s->h_flag[slot] = 0;
  cudaStream_t st = s->s_pub;
  cudaError_t e = cudaMemcpyAsync(s->d_src + a, s->h_src + a, sizeof(pp_source) * r->src.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_off + b, s->h_off + b, sizeof(uint64_t) * r->off.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_chunk + c, s->h_chunk + c, sizeof(uint32_t) * r->chunk.size(),
                        cudaMemcpyHostToDevice, st);
  // outputs cleared by copies of zeros (copy engine, no kernel: the serving
  // kernel may be holding every SM)
  if (e == cudaSuccess && n_dom)
    e = cudaMemcpyAsync(s->d_hits + (size_t)slot * n_dom, s->h_zero, sizeof(uint64_t) * n_dom,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_counts + (size_t)slot * 4, s->h_zero, sizeof(uint64_t) * 4,
                        cudaMemcpyHostToDevice, st);
  // the entry without its claim word, then the claim word (arming the slot
  // only once the rest is in place: a warp still adding to the slot's
  // previous claim word finds the new seq and takes nothing)
  constexpr size_t kWord = sizeof(unsigned long long);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(reinterpret_cast<char*>(s->d_req + slot) + kWord,
                        reinterpret_cast<const char*>(&q) + kWord,
                        sizeof(ppk::ServeReq) - kWord, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->d_req[slot].claimed, s->h_arm + slot, kWord, cudaMemcpyHostToDevice,
                        st);
  // work in flight: the kernel's idle warps must stay
  if (e == cudaSuccess && s->may_leave) {
    e = cudaMemcpyAsync(s->d_may_leave, s->h_zero, sizeof(int), cudaMemcpyHostToDevice, st);
    s->may_leave = false;
  }
  // the doorbell: requests are published in order, so the tail only grows
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_tail, s->h_tail + slot, sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    // a publication cut short would leave a hole in the ring's order: the
    // server stops taking work and fails what it holds
    s->last_error = std::string("publication: ") + cudaGetErrorString(e);
    s->broken = true;
    r->status = PP_ECUDA;
    return true;
  }
  r->status = kPublished;
  s->published += 1;
  return true;
}

// Releases a finished request's slot, arena ranges and budget (lock held).
void release(pp_server* s, Request* r) {
  s->a_src.give(r->src_at, r->src.size());
  s->a_off.give(r->off_at, r->off.size());
  s->a_chunk.give(r->chunk_at, r->chunk.size());
  s->admitted_bytes -= r->bytes;
  s->by_slot[r->slot] = nullptr;
  r->src.clear();
  r->src.shrink_to_fit();
  r->off.clear();
  r->off.shrink_to_fit();
  r->chunk.clear();
  r->chunk.shrink_to_fit();
}

// One pass over the admitted requests (lock held): a raised done flag starts
// the copy of the request's outputs; a finished copy completes the request.
// Returns true when a request completed.
bool poll_admitted(pp_server* s) {
  const int n_dom = s->view.geom.n_dom;
  bool any = false;
  for (int slot = 0; slot < s->cap; ++slot) {
    Request* r = s->by_slot[slot];
    if (!r) continue;
    if (r->status == kPublished && s->h_flag[slot] == (uint32_t)(r->seq + 1)) {
      cudaStream_t st = s->s_down;
      cudaError_t e = cudaSuccess;
      if (n_dom)
        e = cudaMemcpyAsync(s->h_hits + (size_t)slot * n_dom, s->d_hits + (size_t)slot * n_dom,
                            sizeof(uint64_t) * n_dom, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_counts + (size_t)slot * 4, s->d_counts + (size_t)slot * 4,
                            sizeof(uint64_t) * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_err + slot, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaEventRecord(s->copied[slot], st);
      if (e != cudaSuccess) {
        s->last_error = std::string("result copy: ") + cudaGetErrorString(e);
        r->status = PP_ECUDA;
      } else {
        r->status = kCopying;
        continue;
      }
    }
    if (r->status == kCopying) {
      const cudaError_t q = cudaEventQuery(s->copied[slot]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        s->last_error = std::string("result copy: ") + cudaGetErrorString(q);
        r->status = PP_ECUDA;
      } else {
        r->hits.assign(s->h_hits + (size_t)slot * n_dom, s->h_hits + (size_t)(slot + 1) * n_dom);
        std::memcpy(r->counts, s->h_counts + (size_t)slot * 4, sizeof(r->counts));
        r->status = s->h_err[slot] ? PP_EDEVICE : PP_OK;
      }
    }
    if (r->status == kPublished && s->broken) r->status = PP_ECUDA;
    if (r->status <= 0) {  // done or failed
      r->t_done = Clock::now();
      if (r->status == PP_OK) {
        s->latency_ms.push_back(
            std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        s->done_requests += 1;
        s->done_photons += r->n_photons;
        s->t_last_done = r->t_done;
      }
      release(s, r);
      any = true;
    }
  }
  return any;
}

bool unfinished_published(const pp_server* s) {
  for (int slot = 0; slot < s->cap; ++slot) {
    const Request* r = s->by_slot[slot];
    if (r && r->status == kPublished) return true;
  }
  return false;
}

cudaError_t launch_kernel(pp_server* s) {
  ppk::ServeDev sv{};
  sv.req = s->d_req;
  sv.cap = s->cap;
  sv.tail = s->d_tail;
  sv.head = s->d_head;
  sv.src = s->d_src;
  sv.off = s->d_off;
  sv.chunk = s->d_chunk;
  sv.hits = reinterpret_cast<unsigned long long*>(s->d_hits);
  sv.counts = reinterpret_cast<unsigned long long*>(s->d_counts);
  sv.done_flag = s->d_flag;
  sv.err = s->d_err;
  sv.may_leave = s->d_may_leave;
  sv.closing = s->d_closing;
  sv.idle_ns = (uint64_t)s->cfg.idle_exit_us * 1000ull;
  sv.max_ns = (uint64_t)s->cfg.max_launch_ms * 1000000ull;
  ppk::NvtxRange range("pp.server_kernel");
  // a fresh launch is open (a copy of zero: the previous launch has ended)
  cudaError_t e = cudaMemcpyAsync(s->d_closing, s->h_zero, sizeof(int), cudaMemcpyHostToDevice,
                                  s->s_kern);
  if (e == cudaSuccess) e = ppk::launch_serve(s->view.ice, s->view.geom, sv, s->view.run, s->grid, s->smem,
                                    s->s_kern);
  if (e == cudaSuccess) e = cudaEventRecord(s->kern_done, s->s_kern);
  if (e == cudaSuccess) {
    s->kernel_running = true;
    s->launches += 1;
  }
  return e;
}

void scheduler(pp_server* s) {
  cudaSetDevice(s->view.device);  // this library-owned thread works on the server's device
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool woke = false;
    if (poll_admitted(s)) woke = true;
    if (s->broken) {
      while (!s->pending.empty()) {
        s->pending.front()->status = PP_ECUDA;
        s->pending.pop_front();
        woke = true;
      }
    }
    while (!s->broken && !s->pending.empty() && admit_front(s)) {
    }
    if (s->kernel_running) {
      const cudaError_t q = cudaEventQuery(s->kern_done);
      if (q != cudaErrorNotReady) {
        s->kernel_running = false;
        if (q != cudaSuccess) {
          s->last_error = std::string("serving kernel: ") + cudaGetErrorString(q);
          s->broken = true;
        }
      }
    }
    // nothing left on the device: the kernel's idle warps may leave
    if (!s->may_leave && !s->broken && !unfinished_published(s) && s->pending.empty()) {
      const cudaError_t e = cudaMemcpyAsync(s->d_may_leave, s->h_one, sizeof(int),
                                            cudaMemcpyHostToDevice, s->s_pub);
      if (e != cudaSuccess) {
        s->last_error = std::string("serving flag: ") + cudaGetErrorString(e);
        s->broken = true;
      }
      s->may_leave = true;
    }
    if (!s->kernel_running && !s->broken && unfinished_published(s)) {
      const cudaError_t e = launch_kernel(s);
      if (e != cudaSuccess) {
        s->last_error = std::string("serving kernel launch: ") + cudaGetErrorString(e);
        s->broken = true;
      }
    }
    if (woke) s->cv_done.notify_all();
    bool holding = s->kernel_running || !s->pending.empty();
    for (int slot = 0; slot < s->cap && !holding; ++slot) holding = s->by_slot[slot] != nullptr;
    if (s->stop && !holding) break;
    // while work is in flight, look again after a short wait (the device
    // raises done flags in host memory; nothing signals this thread); else
    // sleep until a submission or the stop
    if (holding)
      s->cv_sched.wait_for(lk, std::chrono::microseconds(40));
    else
      s->cv_sched.wait(lk, [&]() { return s->stop || !s->pending.empty(); });
  }
  s->cv_done.notify_all();
}

}  // namespace

extern "C" {

int pp_server_config_default(pp_server_config* cfg) {
  if (!cfg) return PP_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->budget_bytes = 8ull << 30;
  cfg->arena_sources = 1 << 22;
  cfg->ring_requests = 256;
  cfg->idle_exit_us = 1000;
  cfg->max_launch_ms = 200;
  return PP_OK;
}

int pp_server_create(pp_ctx* ctx, const pp_server_config* cfg, pp_server** out) {
  if (!ctx || !cfg || !out) return PP_EINVAL;
  *out = nullptr;
  const int R = cfg->ring_requests;
  if (R < 1 || R > ppk::kServeMaxRequests || (R & (R - 1)) != 0 || cfg->arena_sources < 1 ||
      cfg->arena_sources > ppk::kMaxSources || cfg->budget_bytes == 0 || cfg->idle_exit_us < 0 ||
      cfg->max_launch_ms < 1)
    return PP_EINVAL;
  pp_server* s = new pp_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  s->cap = R;
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
  // the serving kernel: 1024-thread blocks holding the tables and the warps'
  // photon reserves, as many as fit on each SM
  s->smem = ppk::tables_smem_bytes(s->view.ice, s->view.geom) +
            ppk::reserve_smem_bytes(ppk::kServeThreads, false);
  int occ = 0, sms = 0;
  cudaError_t e = ppk::serve_occupancy(s->smem, &occ);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->view.device);
  if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
  s->grid = occ * sms;
  s->by_slot.assign(R, nullptr);
  if (e == cudaSuccess) e = alloc_server_memory(s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    free_server_memory(s);
    ppk::attach_server(ctx, -1);
    delete s;
    return PP_ENOMEM;
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
  if (s->s_kern) cudaStreamSynchronize(s->s_kern);
  if (s->s_pub) cudaStreamSynchronize(s->s_pub);
  if (s->s_down) cudaStreamSynchronize(s->s_down);
  free_server_memory(s);
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
  for (int64_t i = 0; i < n_src; ++i)
    if (!source_ok(src[i])) return PP_EINVAL;
  Request* r = new Request();
  r->event_id = event_id;
  r->src.assign(src, src + n_src);
  expand_on_host(r);
  if (r->n_photons >= ppk::kServeMaxPhotons) {  // room in the claim word's photon field
    delete r;
    return PP_EINVAL;
  }
  r->bytes = request_bytes(s, r);
  if (r->bytes > s->cfg.budget_bytes || n_src > s->cfg.arena_sources) {
    delete r;
    return PP_EBUDGET;
  }
  r->t_submit = Clock::now();
  if (r->n_photons == 0) {  // nothing to propagate: its result is all zeros at once
    r->hits.assign((size_t)s->view.geom.n_dom, 0);
    r->status = PP_OK;
    r->t_done = r->t_submit;
    r->src.clear();
    r->off.clear();
    r->chunk.clear();
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop || s->broken) {
      delete r;
      return s->broken ? PP_ECUDA : PP_EINVAL;
    }
    r->ticket = s->next_ticket++;
    s->by_ticket[r->ticket] = r;
    if (r->status == kQueued) {
      s->pending.push_back(r);
    } else {
      s->latency_ms.push_back(0.0);
      s->done_requests += 1;
    }
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
  auto ready = [&]() { return r->status <= 0; };
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
  out8[5] = (double)s->launches;
  out8[6] = (double)s->peak_bytes;
  out8[7] = (double)s->device_bytes;
  return PP_OK;
}

}  // extern "C"
