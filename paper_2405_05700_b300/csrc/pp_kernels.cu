// Kernels of the photon-propagation path and their launchers.
//
//   a1  source expansion: exclusive prefix of photons per source (u64), the
//       photon-chunk -> first-source table and the source -> event map
//   a2-a7 propagation: one photon per thread (plain), or persistent blocks
//       whose warps refill idle lanes with new photons (a8)
//   debug: Philox blocks, photon traces, hit tests on given segments
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "pp_device.cuh"
#include "pp_internal.h"

namespace ppk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Exclusive block scan of one u64 per thread; returns the thread's prefix and
// the block total.  ws: shared scratch of 32 u64.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* ws,
                                                         uint64_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = (lane < nw) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    ws[lane] = w;
  }
  __syncthreads();
  const uint64_t before = (warp > 0) ? ws[warp - 1] : 0;
  total = ws[nw - 1];
  __syncthreads();
  return before + x - v;
}

__device__ __forceinline__ uint32_t chunk_log2_for(uint64_t total, int64_t n_src) {
  uint32_t k = 0;
  const uint64_t cap = (uint64_t)(n_src > 0 ? n_src : 1);
  while ((total >> k) > cap) ++k;
  return k;
}

// Event slot of source s: last e with src_begin[e] <= s (and a non-empty range).
__device__ __forceinline__ uint32_t event_of(const int64_t* src_begin, int n_events, int64_t s) {
  int lo = 0, hi = n_events - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (src_begin[mid] <= s) lo = mid;
    else hi = mid - 1;
  }
  return (uint32_t)lo;
}

// Chunk c of 2^k photons starts in source upper_bound(off, c 2^k) - 1.
__device__ __forceinline__ void chunk_entry(const uint64_t* off, int64_t n_src, uint64_t c,
                                            uint32_t k, uint32_t* chunk_src) {
  const uint64_t g = c << k;
  int64_t lo = 0, hi = n_src - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  chunk_src[c] = (uint32_t)lo;
}

// ---- a1, small batches: one block does scan, maps and chunk table ----------
// Per-source event record: event slot, event-local photon base, event id.
__device__ __forceinline__ void write_aux(const uint64_t* off, const int64_t* src_begin,
                                          const uint64_t* event_ids, int n_events, int64_t s,
                                          SrcAux* aux) {
  const uint32_t e = event_of(src_begin, n_events, s);
  SrcAux a;
  a.base = off[s] - off[src_begin[e]];
  a.ev_lo = (uint32_t)event_ids[e];
  a.ev = e;
  aux[s] = a;
}

__global__ void __launch_bounds__(kSmallThreads)
k_expand_small(const pp_source* __restrict__ src, int64_t n_src,
               const int64_t* __restrict__ src_begin, const uint64_t* __restrict__ event_ids,
               int n_events, ExpandBufs b) {
  __shared__ uint64_t ws[32];
  __shared__ uint64_t s_total;
  __shared__ uint32_t s_k;
  const int64_t base = (int64_t)threadIdx.x * kSmallItems;
  uint64_t v[kSmallItems];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kSmallItems; ++i) {
    const int64_t s = base + i;
    v[i] = (s < n_src) ? src[s].n_photons : 0;
    sum += v[i];
  }
  uint64_t total;
  uint64_t pre = block_exclusive_scan(sum, ws, total);
#pragma unroll
  for (int i = 0; i < kSmallItems; ++i) {
    const int64_t s = base + i;
    if (s < n_src) b.off[s] = pre;
    pre += v[i];
  }
  if (threadIdx.x == 0) {
    b.off[n_src] = total;
    s_total = total;
    s_k = chunk_log2_for(total, n_src);
    b.meta[0] = total;
    b.meta[1] = s_k;
  }
  __syncthreads();  // off[] written by this block is visible to it after the barrier
  const uint64_t n_chunks = (s_total + (1ull << s_k) - 1) >> s_k;
  for (uint64_t c = threadIdx.x; c <= n_chunks; c += blockDim.x)
    chunk_entry(b.off, n_src, c, s_k, b.chunk_src);
  if (b.aux)
    for (int64_t s = threadIdx.x; s < n_src; s += blockDim.x)
      write_aux(b.off, src_begin, event_ids, n_events, s, b.aux);
}

// ---- a1, large batches: partial sums, top scan, final pass, chunk table ----
__global__ void __launch_bounds__(kScanThreads)
k_scan_partial(const pp_source* __restrict__ src, int64_t n_src, uint64_t* __restrict__ bsum) {
  __shared__ uint64_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n_src) sum += src[base + i].n_photons;
  uint64_t total;
  block_exclusive_scan(sum, ws, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kTopThreads)
k_scan_top(uint64_t* __restrict__ bsum, int nb, int64_t n_src, uint64_t* __restrict__ meta) {
  __shared__ uint64_t ws[32];
  const int base = threadIdx.x * kTopItems;
  uint64_t v[kTopItems];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kTopItems; ++i) {
    v[i] = (base + i < nb) ? bsum[base + i] : 0;
    sum += v[i];
  }
  uint64_t total;
  uint64_t pre = block_exclusive_scan(sum, ws, total);
#pragma unroll
  for (int i = 0; i < kTopItems; ++i) {
    if (base + i < nb) bsum[base + i] = pre;
    pre += v[i];
  }
  if (threadIdx.x == 0) {
    meta[0] = total;
    meta[1] = chunk_log2_for(total, n_src);
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_final(const pp_source* __restrict__ src, int64_t n_src,
             const uint64_t* __restrict__ bsum, ExpandBufs b) {
  __shared__ uint64_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n_src) ? src[base + i].n_photons : 0;
    sum += v[i];
  }
  uint64_t total;
  uint64_t pre = block_exclusive_scan(sum, ws, total) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t s = base + i;
    if (s < n_src) b.off[s] = pre;
    pre += v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) b.off[n_src] = b.meta[0];
}

// Chunk table and per-source event records, once all offsets are known.
__global__ void k_finish(int64_t n_src, const int64_t* __restrict__ src_begin,
                         const uint64_t* __restrict__ event_ids, int n_events, ExpandBufs b) {
  const uint64_t total = b.meta[0];
  const uint32_t k = (uint32_t)b.meta[1];
  const uint64_t n_chunks = (total + (1ull << k) - 1) >> k;
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c <= n_chunks) chunk_entry(b.off, n_src, c, k, b.chunk_src);
  if (b.aux && (int64_t)c < n_src) write_aux(b.off, src_begin, event_ids, n_events, (int64_t)c, b.aux);
}

// ---- a2..a8: propagation ---------------------------------------------------
__device__ __forceinline__ void flush_path_stats(const WorkDev& W, uint64_t steps,
                                                 uint32_t crossings, uint32_t births,
                                                 uint32_t slow) {
  if (!W.stats) return;
  unsigned long long v0 = steps, v1 = crossings, v2 = births, v3 = slow;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(kFull, v0, o);
    v1 += __shfl_down_sync(kFull, v1, o);
    v2 += __shfl_down_sync(kFull, v2, o);
    v3 += __shfl_down_sync(kFull, v3, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(W.stats + 0, v0);
    atomicAdd(W.stats + 1, v1);
    atomicAdd(W.stats + 2, v2);
    atomicAdd(W.stats + 3, v3);
  }
}

// a8 with a photon reserve: the warp keeps up to kReserveCap born photons in
// shared memory.  Whenever the reserve holds no more than kReserveCap - 32,
// the warp claims 32 photon indices with one atomic and all 32 lanes give
// birth together (one converged pass, instead of a pass for the few lanes
// that happen to be idle); idle lanes take the next reserved photons once
// `refill` of them are idle (or the work is exhausted).  Only which lane runs
// which photon changes: every photon still draws its own Philox streams.
// Values the reserve loop needs only at a top-up or a hand-out are re-read
// there instead of being kept in registers across the photon step (whose
// register budget is what limits the kernel): special registers and the
// expansion's totals, read with volatile asm so that the compiler does not
// hoist them out of the loop.
extern __shared__ __align__(16) unsigned char dyn_smem[];

__device__ __forceinline__ unsigned tid_x() {
  unsigned t;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
  return t;
}

__device__ __forceinline__ unsigned lanes_below() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t ld_u64_volatile(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// The warp's reserve ring, after the tables.
template <bool kRecords>
__device__ __forceinline__ uint32_t* reserve_ring(const IceDev& I, const GeomDev& G) {
  constexpr int RW = kRecords ? kReserveWordsRecords : kReserveWords;
  uint32_t* rings = reinterpret_cast<uint32_t*>(dyn_smem + tables_bytes(I.L, G.n_str, G.nx * G.ny));
  return rings + (tid_x() >> 5) * (kReserveCap * RW);
}

// A born photon into ring slot `slot` / the photon of a slot out of the ring
// (word-major: word j of slot i at ring[j * kReserveCap + i]).
template <bool kRecords>
__device__ __forceinline__ void ring_put(uint32_t* ring, int slot, const Photon& q, int src) {
  constexpr int CAP = kReserveCap;
  float* ringf = reinterpret_cast<float*>(ring);
  ringf[0 * CAP + slot] = q.px;
  ringf[1 * CAP + slot] = q.py;
  ringf[2 * CAP + slot] = q.pz;
  ringf[3 * CAP + slot] = q.dx;
  ringf[4 * CAP + slot] = q.dy;
  ringf[5 * CAP + slot] = q.dz;
  ringf[6 * CAP + slot] = q.tau_a;
  ring[7 * CAP + slot] = (uint32_t)q.layer;
  ring[8 * CAP + slot] = q.pid_lo;
  ring[9 * CAP + slot] = q.pid_hi;
  ring[10 * CAP + slot] = q.ev_lo;
  ring[11 * CAP + slot] = (uint32_t)q.ev;
  if (kRecords) {
    ringf[12 * CAP + slot] = q.t_emit;
    ring[13 * CAP + slot] = (uint32_t)src;
  }
}

template <bool kRecords>
__device__ __forceinline__ void ring_take(const uint32_t* ring, int slot, Photon& ph) {
  constexpr int CAP = kReserveCap;
  const float* ringf = reinterpret_cast<const float*>(ring);
  ph.px = ringf[0 * CAP + slot];
  ph.py = ringf[1 * CAP + slot];
  ph.pz = ringf[2 * CAP + slot];
  ph.dx = ringf[3 * CAP + slot];
  ph.dy = ringf[4 * CAP + slot];
  ph.dz = ringf[5 * CAP + slot];
  ph.tau_a = ringf[6 * CAP + slot];
  ph.layer = (int)ring[7 * CAP + slot];
  ph.pid_lo = ring[8 * CAP + slot];
  ph.pid_hi = ring[9 * CAP + slot];
  ph.ev_lo = ring[10 * CAP + slot];
  ph.ev = (int)ring[11 * CAP + slot];
  if (kRecords) {
    ph.t_emit = ringf[12 * CAP + slot];
    ph.src = (int)ring[13 * CAP + slot];
  }
  ph.path = 0.0f;
  ph.n = 0;
  ph.cb = -1.0f;
}

// One top-up of the warp's reserve: claim 32 photon indices with one atomic,
// give birth to them on all 32 lanes, append the well-formed ones to the ring
// after its rcount live slots from rhead.  Returns the new rcount; sets
// `exhausted` once the claim reaches the end of the work.  Kept out of line:
// it runs once per ~40 steps of the warp, and as a call its temporaries do
// not compete for registers with the photon step.
template <bool kRecords>
__device__ __noinline__ int topup(const IceDev& I, const GeomDev& G, const WorkDev& W,
                                  const RunDev& R, int rhead, int rcount, bool& exhausted) {
  constexpr int CAP = kReserveCap;
  const uint64_t total = ld_u64_volatile(W.meta + 0);
  const uint32_t k = (uint32_t)ld_u64_volatile(W.meta + 1);
  const uint64_t end = total < W.g_end ? total : W.g_end;
  const unsigned lane = tid_x() & 31;
  unsigned long long base = 0;
  if (lane == 0) base = W.g_begin + atomicAdd(W.work, 32ull);
  base = __shfl_sync(kFull, base, 0);
  if (base + 32 >= end) exhausted = true;
  if (base < end) {
    uint64_t in_src = 0;
    const int s = locate_claim(W, k, base, lane, end, in_src);
    const uint64_t g = base + lane;
    bool ok = false;
    Photon q;
    if (g < end) {
      identify(W, s, in_src, g, q);
      ok = birth(q, W.src[s], I, R);
      if (!ok) atomicOr(W.err, kErrBadSource);
    }
    const unsigned okm = __ballot_sync(kFull, ok);
    if (W.stats && lane == 0) {
      const uint64_t left = end - base;
      atomicAdd(W.stats + 2, (unsigned long long)(left < 32 ? left : 32));
    }
    if (ok) {
      int slot = rhead + rcount + __popc(okm & lanes_below());
      if (slot >= CAP) slot -= CAP;
      ring_put<kRecords>(reserve_ring<kRecords>(I, G), slot, q, s);
    }
    rcount += __popc(okm);
  }
  return rcount;
}

template <bool kRecords>
__device__ __forceinline__ void run_with_reserve(const IceDev& I, const GeomDev& G,
                                                 const WorkDev& W, const RunDev& R,
                                                 const Tables& T) {
  constexpr int CAP = kReserveCap;
  bool alive = false, exhausted = false;
  int rhead = 0, rcount = 0;  // warp-uniform ring state
  // path statistics: births are added per warp at each top-up; steps per lane
  // fit 32 bits (a launch gives a lane far fewer than 2^32 steps)
  uint32_t crossings = 0, slow = 0, steps = 0;
  LaneTally lt;
  Photon ph;
  for (;;) {
    if (!exhausted && rcount <= CAP - 32) {
      __syncwarp();  // earlier reads of the slots about to be refilled are done
      rcount = topup<kRecords>(I, G, W, R, rhead, rcount, exhausted);
      __syncwarp();  // the new slots are visible to every lane of the warp
    }
    const unsigned idle = __ballot_sync(kFull, !alive);
    const int n_idle = __popc(idle);
    if (rcount > 0 && n_idle > 0 && (n_idle >= R.refill || exhausted)) {
      const int n = min(n_idle, rcount);
      const int rank = __popc(idle & lanes_below());
      if (!alive && rank < n) {
        int slot = rhead + rank;
        if (slot >= CAP) slot -= CAP;
        ring_take<kRecords>(reserve_ring<kRecords>(I, G), slot, ph);
        alive = true;
      }
      rhead += n;
      if (rhead >= CAP) rhead -= CAP;
      rcount -= n;
    }
    if (__ballot_sync(kFull, alive) == 0) {
      if (exhausted && rcount == 0) break;
      continue;
    }
    if (alive) {
      const int out = photon_step(ph, I, G, T, R, crossings, slow);
      if (out != kScattered) {
        tally(W, G.n_dom, ph, out, lt);
        if (kRecords && out >= 0) record_hit(W, R, ph, out);
        steps += ph.n;
        alive = false;
      }
    }
  }
  flush(W, lt);
  flush_path_stats(W, steps, crossings, 0, slow);
}

// kRecords (persistent only): also append a compact record per hit.
// kReserve (persistent only): the photon reserve above.
template <bool kPersistent, int kMinBlocks, bool kRecords = false, bool kReserve = false>
__global__ void __launch_bounds__(kMinBlocks > 0 ? 256 : 1024, kMinBlocks > 0 ? kMinBlocks : 1)
k_propagate(const __grid_constant__ IceDev I, const __grid_constant__ GeomDev G,
            const __grid_constant__ WorkDev W, const __grid_constant__ RunDev R, uint64_t n_plain) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tables T = stage_tables(smem, I, G);
  __syncthreads();
  const uint64_t total = __ldg(W.meta + 0);
  const uint32_t k = (uint32_t)__ldg(W.meta + 1);
  if (kPersistent && kReserve) {
    run_with_reserve<kRecords>(I, G, W, R, T);
    return;
  }
  Photon ph;
  if (!kPersistent) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total || g >= n_plain) return;
    const int s = locate(W, k, g, ph);
    const pp_source src = W.src[s];
    if (!birth(ph, src, I, R)) {
      atomicOr(W.err, kErrBadSource);
      return;
    }
    uint32_t crossings = 0, slow = 0;
    for (;;) {
      const int out = photon_step(ph, I, G, T, R, crossings, slow);
      if (out != kScattered) {
        tally(W, G.n_dom, ph, out);
        return;
      }
    }
  } else {
    // a8: each warp keeps its 32 lanes busy; once `refill` lanes are idle the
    // warp claims that many consecutive photon indices with one atomic.
    const unsigned lane = threadIdx.x & 31;
    bool alive = false;
    bool exhausted = false;
    uint32_t crossings = 0, births = 0, slow = 0;
    uint64_t steps = 0;
    LaneTally lt;
    // photons [g_begin, end) of the batch: claims count from g_begin
    const uint64_t end = total < W.g_end ? total : W.g_end;
    for (;;) {
      const unsigned idle = __ballot_sync(kFull, !alive);
      const int n_idle = __popc(idle);
      if (!exhausted && n_idle >= R.refill) {
        unsigned long long base = 0;
        if (lane == 0) base = W.g_begin + atomicAdd(W.work, (unsigned long long)n_idle);
        base = __shfl_sync(kFull, base, 0);
        if (base + (unsigned long long)n_idle >= end) exhausted = true;
        if (base < end) {
          const uint32_t rank = __popc(idle & ((1u << lane) - 1u));
          uint64_t in_src = 0;
          const int s = locate_claim(W, k, base, rank, end, in_src);
          const uint64_t g = base + rank;
          if (!alive && g < end) {
            identify(W, s, in_src, g, ph);
            const pp_source src = W.src[s];
            alive = birth(ph, src, I, R);
            if (kRecords) ph.src = s;
            births += 1;
            if (!alive) atomicOr(W.err, kErrBadSource);
          }
        }
      }
      if (__ballot_sync(kFull, alive) == 0) {
        if (exhausted) break;
        continue;
      }
      if (alive) {
        const int out = photon_step(ph, I, G, T, R, crossings, slow);
        if (out != kScattered) {
          tally(W, G.n_dom, ph, out, lt);
          if (kRecords && out >= 0) record_hit(W, R, ph, out);
          steps += ph.n;
          alive = false;
        }
      }
    }
    flush(W, lt);
    flush_path_stats(W, steps, crossings, births, slow);
  }
}

// ---- serving: photons pulled from the device request ring -------------------
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Per-lane tallies of the request the lane last worked on (as LaneTally),
// plus the number of its photons tallied.  The flush adds them to the
// request's counters and that number to its done count, after a fence that
// makes the lane's hit atomics visible first; the flush that brings done to
// the request's total raises the request's host-visible flag.
struct ServeTally {
  int slot = -1;
  uint32_t absorbed = 0, escaped = 0, truncated = 0, photons = 0;
  unsigned long long steps = 0;
};

__device__ __forceinline__ void serve_done(const ServeDev& S, int slot, unsigned long long n) {
  __threadfence();
  ServeReq* r = S.req + slot;
  const unsigned long long before = atomicAdd(&r->done, n);
  if (before + n == __ldcg(&r->total)) {
    __threadfence_system();
    S.done_flag[slot] = __ldcg(&r->seq) + 1u;
  }
}

__device__ __noinline__ void serve_flush(const ServeDev& S, ServeTally& t) {
  if (t.slot >= 0 && t.photons) {
    unsigned long long* cnt = S.counts + (size_t)t.slot * 4;
    if (t.absorbed) atomicAdd(cnt + 0, (unsigned long long)t.absorbed);
    if (t.escaped) atomicAdd(cnt + 1, (unsigned long long)t.escaped);
    if (t.truncated) atomicAdd(cnt + 2, (unsigned long long)t.truncated);
    if (t.steps) atomicAdd(cnt + 3, t.steps);
    serve_done(S, t.slot, t.photons);
  }
  t = ServeTally();
}

__device__ __forceinline__ void serve_tally(const ServeDev& S, int n_dom, const Photon& ph,
                                            int out, ServeTally& t) {
  if (ph.ev != t.slot) {
    serve_flush(S, t);
    t.slot = ph.ev;
  }
  if (out >= 0) {
    atomicAdd(S.hits + (size_t)ph.ev * n_dom + out, 1ull);
  } else if (out == kEscaped) {
    t.escaped += 1;
  } else {
    t.absorbed += 1;
    if (out == kTruncated) t.truncated += 1;
  }
  t.photons += 1;
  t.steps += ph.n;
}

// One top-up of the warp's reserve from the request ring: lane 0 claims up to
// 32 photons of the oldest request with unclaimed photons (one atomic add to
// its slot's claim word; moving the shared head past a request whose photons
// are all claimed), all lanes give birth to them and append them to the ring.
// The photon's event slot is the request's ring slot, so that its tallies go
// to that request's outputs.  `got` is false when no published request has
// unclaimed photons.
__device__ __noinline__ int serve_topup(const IceDev& I, const GeomDev& G, const ServeDev& S,
                                        const RunDev& R, int rhead, int rcount, bool& got) {
  constexpr int CAP = kReserveCap;
  constexpr unsigned long long kOffMask = (1ull << kServeOffsetBits) - 1ull;
  constexpr unsigned kSeqMask = (1u << kServeSeqBits) - 1u;
  const unsigned lane = tid_x() & 31;
  unsigned long long o = 0, tot = 0, src_off = 0, off_off = 0, chunk_off = 0;
  unsigned n_src = 0, k = 0, ev_lo = 0, slot_req = 0;
  int ok_claim = 0;
  if (lane == 0) {
    for (int tries = 0; tries < 64; ++tries) {
      const unsigned long long h = ld_relaxed(S.head);
      if (h >= ld_relaxed(S.tail)) break;  // every published photon is claimed
      slot_req = (unsigned)(h & (unsigned long long)(S.cap - 1));
      ServeReq* r = S.req + slot_req;
      const unsigned long long c = atomicAdd(&r->claimed, 32ull);
      const unsigned seq_c = (unsigned)(c >> kServeOffsetBits);
      o = c & kOffMask;
      // the slot's entry was written by host copies: read it through L2,
      // after the claim (and the seq after the total: if the slot was
      // rewritten meanwhile, the seq no longer matches the claim's)
      __threadfence();
      tot = __ldcg(&r->total);
      __threadfence();
      const unsigned sq = __ldcg(&r->seq) & kSeqMask;
      if (sq != seq_c) continue;  // a claim on the slot's previous request: nothing taken
      if (o >= tot) {             // every photon of this request is claimed
        atomicCAS(S.head, h, h + 1);
        continue;
      }
      src_off = __ldcg(&r->src_off);
      off_off = __ldcg(&r->off_off);
      chunk_off = __ldcg(&r->chunk_off);
      n_src = __ldcg(&r->n_src);
      k = __ldcg(&r->chunk_log2);
      ev_lo = __ldcg(&r->event_lo);
      ok_claim = 1;
      break;
    }
  }
  got = __shfl_sync(kFull, ok_claim, 0) != 0;
  if (!got) return rcount;
  o = __shfl_sync(kFull, o, 0);
  tot = __shfl_sync(kFull, tot, 0);
  if (tot - o > 32ull) tot = o + 32ull;  // this claim's photons end here
  slot_req = __shfl_sync(kFull, slot_req, 0);
  WorkDev Wv{};
  Wv.src = S.src + __shfl_sync(kFull, src_off, 0);
  Wv.off = S.off + __shfl_sync(kFull, off_off, 0);
  Wv.chunk_src = S.chunk + __shfl_sync(kFull, chunk_off, 0);
  Wv.aux = nullptr;
  Wv.n_src = (int)__shfl_sync(kFull, n_src, 0);
  Wv.single_event_lo = __shfl_sync(kFull, ev_lo, 0);
  k = __shfl_sync(kFull, k, 0);
  uint64_t in_src = 0;
  const int s = locate_claim<true>(Wv, k, o, lane, tot, in_src);
  const uint64_t g = o + lane;
  bool ok = false;
  Photon q;
  if (g < tot) {
    identify(Wv, s, in_src, g, q);
    q.ev = (int)slot_req;
    // the source record, also through L2 (the arena range may have held
    // another request's sources)
    pp_source src;
    const uint2* sp = reinterpret_cast<const uint2*>(Wv.src + s);
    uint2* dp = reinterpret_cast<uint2*>(&src);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(pp_source) / sizeof(uint2)); ++w) dp[w] = __ldcg(sp + w);
    ok = birth(q, src, I, R);
    if (!ok) {  // a malformed source (the host checks them): raise the error, count it done
      atomicOr(S.err, kErrBadSource);
      serve_done(S, (int)slot_req, 1);
    }
  }
  const unsigned okm = __ballot_sync(kFull, ok);
  if (ok) {
    int slot = rhead + rcount + __popc(okm & lanes_below());
    if (slot >= CAP) slot -= CAP;
    ring_put<false>(reserve_ring<false>(I, G), slot, q, s);
  }
  return rcount + __popc(okm);
}

// The serving kernel: the reserve loop of the batched kernel, fed from the
// request ring.  A warp keeps taking photons while requests are published;
// once it has nothing in flight and nothing to claim it polls (sleeping a few
// microseconds between looks).  A launch ends as a whole: a warp that has
// been idle for idle_ns while the host holds no unfinished request
// (may_leave), or any warp max_ns after the launch, closes it (`closing`);
// then no warp claims again and every warp leaves once its photons are done.
// (Warps leaving one by one would leave the next request to the few still
// running.)  Every wait is bounded by the global timer; the host relaunches
// the kernel while published requests are unfinished.
__global__ void __launch_bounds__(kServeThreads, 1)
k_serve(const __grid_constant__ IceDev I, const __grid_constant__ GeomDev G,
        const __grid_constant__ ServeDev S, const __grid_constant__ RunDev R) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tables T = stage_tables(smem, I, G);
  __syncthreads();
  constexpr int CAP = kReserveCap;
  const uint64_t t0 = __shfl_sync(kFull, global_ns(), 0);
  uint64_t idle_since = 0;
  bool alive = false, claiming = true, idle = false;
  int rhead = 0, rcount = 0;
  uint32_t crossings = 0, slow = 0;
  ServeTally st;
  Photon ph;
  for (;;) {
    bool got = false;
    if (claiming && rcount <= CAP - 32) {
      // once any warp has closed the launch, no warp claims any more
      if (__shfl_sync(kFull, ld_relaxed_int(S.closing), 0)) {
        claiming = false;
      } else {
        __syncwarp();
        rcount = serve_topup(I, G, S, R, rhead, rcount, got);
        __syncwarp();
        const uint64_t now = __shfl_sync(kFull, global_ns(), 0);
        if (now - t0 > S.max_ns) {
          claiming = false;
          if ((threadIdx.x & 31) == 0) atomicExch(S.closing, 1);
        }
        if (got) idle = false;
      }
    }
    const unsigned idle_lanes = __ballot_sync(kFull, !alive);
    const int n_idle = __popc(idle_lanes);
    if (rcount > 0 && n_idle > 0 && (n_idle >= R.refill || !got)) {
      const int n = min(n_idle, rcount);
      const int rank = __popc(idle_lanes & lanes_below());
      if (!alive && rank < n) {
        int slot = rhead + rank;
        if (slot >= CAP) slot -= CAP;
        ring_take<false>(reserve_ring<false>(I, G), slot, ph);
        alive = true;
      }
      rhead += n;
      if (rhead >= CAP) rhead -= CAP;
      rcount -= n;
    }
    // a lane left without a photon hands in its tallies, so that the request
    // it worked on completes as soon as its last photon is done
    if (!alive && st.slot >= 0) serve_flush(S, st);
    if (__ballot_sync(kFull, alive) == 0) {
      if (rcount > 0) continue;
      if (!claiming) break;
      const uint64_t now = __shfl_sync(kFull, global_ns(), 0);
      if (!idle) {
        idle = true;
        idle_since = now;
      }
      const int leave = __shfl_sync(kFull, ld_relaxed_int(S.may_leave), 0);
      if (leave && now - idle_since > S.idle_ns) {
        // the host holds nothing unfinished: close the whole launch (every
        // warp leaves, so that the next request finds a full launch)
        if ((threadIdx.x & 31) == 0) atomicExch(S.closing, 1);
        break;
      }
      __nanosleep(4000);
      continue;
    }
    if (alive) {
      const int out = photon_step(ph, I, G, T, R, crossings, slow);
      if (out != kScattered) {
        serve_tally(S, G.n_dom, ph, out, st);
        alive = false;
      }
    }
  }
  serve_flush(S, st);
}

// ---- debug kernels ---------------------------------------------------------
__global__ void k_trace(IceDev I, GeomDev G, WorkDev W, RunDev R, const uint64_t* ids, int64_t n,
                        int n_trace, int* outcome, int64_t* n_steps, float* birth_out,
                        float* trace) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tables T = stage_tables(smem, I, G);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t total = W.meta[0];
  const uint32_t k = (uint32_t)W.meta[1];
  float* tr = trace ? trace + (size_t)i * n_trace * 3 : nullptr;
  for (int q = 0; tr && q < 3 * n_trace; ++q) tr[q] = __int_as_float(0x7fc00000);
  const uint64_t g = ids[i];
  if (g >= total) {
    outcome[i] = -4;
    n_steps[i] = 0;
    return;
  }
  Photon ph;
  const int s = locate(W, k, g, ph);
  if (!birth(ph, W.src[s], I, R)) {
    outcome[i] = -5;
    n_steps[i] = 0;
    return;
  }
  if (birth_out) {
    float* b = birth_out + (size_t)i * 6;
    b[0] = ph.px; b[1] = ph.py; b[2] = ph.pz;
    b[3] = ph.dx; b[4] = ph.dy; b[5] = ph.dz;
  }
  uint32_t crossings = 0, slow = 0;
  for (;;) {
    const int out = photon_step(ph, I, G, T, R, crossings, slow);
    if ((out == kScattered || out == kTruncated) && tr && (int)ph.n <= n_trace) {
      tr[3 * (ph.n - 1) + 0] = ph.px;
      tr[3 * (ph.n - 1) + 1] = ph.py;
      tr[3 * (ph.n - 1) + 2] = ph.pz;
    }
    if (out != kScattered) {
      outcome[i] = out;
      n_steps[i] = ph.n;
      return;
    }
  }
}

__global__ void k_philox(const uint4* ctr, const uint2* key, uint4* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key[i]);
}

__global__ void k_scatter(IceDev I, const float* dir, const uint32_t* words, float* out,
                          int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float dx = dir[3 * i], dy = dir[3 * i + 1], dz = dir[3 * i + 2];
  float mu, st;
  hg_angle(I, u01f(words[2 * i]), mu, st);
  rotate(dx, dy, dz, mu, st, u01f(words[2 * i + 1]));
  out[3 * i] = dx;
  out[3 * i + 1] = dy;
  out[3 * i + 2] = dz;
}

__global__ void k_first_hit(GeomDev G, IceDev I, const float* seg, int64_t n, int mode, int* dom,
                            float* t) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tables T = stage_tables(smem, I, G);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* q = seg + 7 * i;
  float th;
  uint32_t slow = 0;
  const int k = mode == 0 ? first_hit_grid(G, T, q[0], q[1], q[2], q[3], q[4], q[5], q[6], th, slow)
                          : first_hit_brute(G, q[0], q[1], q[2], q[3], q[4], q[5], q[6], th);
  dom[i] = k;
  t[i] = th;
}

}  // namespace

size_t tables_smem_bytes(const IceDev& ice, const GeomDev& geom) {
  return tables_bytes(ice.L, geom.n_str, geom.nx * geom.ny);
}

cudaError_t launch_expand(const pp_source* src, int64_t n_src, const int64_t* src_begin,
                          const uint64_t* event_ids, int n_events, const ExpandBufs& b,
                          cudaStream_t st) {
  if (n_src <= kSmallMax) {
    k_expand_small<<<1, kSmallThreads, 0, st>>>(src, n_src, src_begin, event_ids, n_events, b);
    return cudaGetLastError();
  }
  const int nb = (int)((n_src + kScanTile - 1) / kScanTile);
  k_scan_partial<<<nb, kScanThreads, 0, st>>>(src, n_src, b.bsum);
  k_scan_top<<<1, kTopThreads, 0, st>>>(b.bsum, nb, n_src, b.meta);
  k_scan_final<<<nb, kScanThreads, 0, st>>>(src, n_src, b.bsum, b);
  const int64_t nc = n_src + 2;
  k_finish<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(n_src, src_begin, event_ids, n_events, b);
  return cudaGetLastError();
}

// The dynamic shared-memory limit is an attribute of each kernel, shared by
// every context on the device: it is only ever raised, so that one context
// cannot lower it under another's launches.
namespace {
std::mutex g_smem_mu;
size_t g_smem_limit[64] = {};
}  // namespace

cudaError_t set_propagate_smem_limit(size_t smem) {
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  if (smem <= g_smem_limit[dev]) return cudaSuccess;
  const void* fns[] = {(const void*)k_propagate<true, 0>, (const void*)k_propagate<true, 5>,
                       (const void*)k_propagate<true, 6>, (const void*)k_propagate<false, 0>,
                       (const void*)k_propagate<true, 0, true>,
                       (const void*)k_propagate<true, 0, false, true>,
                       (const void*)k_propagate<true, 5, false, true>,
                       (const void*)k_propagate<true, 6, false, true>,
                       (const void*)k_propagate<true, 3, false, true>,
                       (const void*)k_propagate<true, 0, true, true>};
  cudaError_t e;
  for (const void* f : fns) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_first_hit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) g_smem_limit[dev] = smem;
  return e;
}

// The kernel instance of a variant (register budget, records, reserve).
const void* propagate_fn(int variant) {
  switch (variant) {
    case 5: return (const void*)k_propagate<true, 5>;
    case 6: return (const void*)k_propagate<true, 6>;
    case kVariantRecords: return (const void*)k_propagate<true, 0, true>;
    case kVariantReserve: return (const void*)k_propagate<true, 0, false, true>;
    case kVariantReserve + 5: return (const void*)k_propagate<true, 5, false, true>;
    case kVariantReserve + 6: return (const void*)k_propagate<true, 6, false, true>;
    case kVariantReserve + 3: return (const void*)k_propagate<true, 3, false, true>;
    case kVariantReserve + kVariantRecords: return (const void*)k_propagate<true, 0, true, true>;
    default: return (const void*)k_propagate<true, 0>;
  }
}

// Register-capped variants (minimum blocks per SM in their launch bounds) run
// 256-thread blocks.
int variant_threads(int variant, int block_threads) {
  const int base = variant % kVariantReserve;
  return (base == 3 || base == 5 || base == 6) ? 256 : block_threads;
}

cudaError_t propagate_occupancy(int block_threads, size_t smem, int variant, int* blocks_per_sm) {
  const int bt = variant_threads(variant, block_threads);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, propagate_fn(variant), bt,
                                                       smem);
}

cudaError_t launch_propagate(bool persistent, const IceDev& ice, const GeomDev& geom,
                             const WorkDev& work, const RunDev& run, int block_threads,
                             int grid_blocks, uint64_t n_photons_host, size_t smem,
                             cudaStream_t st, int variant) {
  if (persistent) {
    const int bt = variant_threads(variant, block_threads);
    void* args[] = {(void*)&ice, (void*)&geom, (void*)&work, (void*)&run, (void*)&n_photons_host};
    return cudaLaunchKernel(propagate_fn(variant), dim3(grid_blocks), dim3(bt), args, smem, st);
  }
  if (n_photons_host == 0) return cudaSuccess;
  const uint64_t nb = (n_photons_host + block_threads - 1) / block_threads;
  k_propagate<false, 0><<<(unsigned)nb, block_threads, smem, st>>>(ice, geom, work, run,
                                                                    n_photons_host);
  return cudaGetLastError();
}

cudaError_t serve_occupancy(size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_serve, kServeThreads, smem);
}

cudaError_t launch_serve(const IceDev& ice, const GeomDev& geom, const ServeDev& sv,
                         const RunDev& run, int grid_blocks, size_t smem, cudaStream_t st) {
  k_serve<<<grid_blocks, kServeThreads, smem, st>>>(ice, geom, sv, run);
  return cudaGetLastError();
}

cudaError_t launch_trace(const IceDev& ice, const GeomDev& geom, const WorkDev& work,
                         const RunDev& run, const uint64_t* ids, int64_t n, int n_trace,
                         int* outcome, int64_t* n_steps, float* birth, float* trace,
                         size_t smem, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_trace<<<(unsigned)((n + 127) / 128), 128, smem, st>>>(ice, geom, work, run, ids, n, n_trace,
                                                          outcome, n_steps, birth, trace);
  return cudaGetLastError();
}

// Host-API argument check on the device: the lowest index of a malformed
// source (non-finite field, zero direction, negative length, unknown type).
__global__ void k_check_sources(const pp_source* __restrict__ src, int64_t n, int64_t base,
                                unsigned long long* first_bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const pp_source s = src[i];
  const bool ok = isfinite(s.x) && isfinite(s.y) && isfinite(s.z) && isfinite(s.dx) &&
                  isfinite(s.dy) && isfinite(s.dz) && isfinite(s.length) && s.length >= 0.0f &&
                  (s.dx != 0.0f || s.dy != 0.0f || s.dz != 0.0f) && s.type <= PP_SRC_CASCADE;
  if (!ok) atomicMin(first_bad, (unsigned long long)(base + i));
}

cudaError_t launch_check_sources(const pp_source* src, int64_t n, int64_t base,
                                 unsigned long long* first_bad, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_check_sources<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, n, base, first_bad);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(ctr), reinterpret_cast<const uint2*>(key),
      reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const IceDev& ice, const float* dir, const uint32_t* words, float* out,
                           int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ice, dir, words, out, n);
  return cudaGetLastError();
}

cudaError_t launch_first_hit(const GeomDev& geom, const IceDev& ice, const float* seg, int64_t n,
                             int mode, int* dom, float* t, size_t smem, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_first_hit<<<(unsigned)((n + 255) / 256), 256, smem, st>>>(geom, ice, seg, n, mode, dom, t);
  return cudaGetLastError();
}

}  // namespace ppk
