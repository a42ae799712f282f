// Kernels of the photon-propagation path and their launchers.
//
//   a1  source expansion: exclusive prefix of photons per source (u64), the
//       photon-chunk -> first-source table and the source -> event map
//   a2-a7 propagation: one photon per thread (plain), or persistent blocks
//       whose warps refill idle lanes with new photons (a8)
//   debug: Philox blocks, photon traces, hit tests on given segments
#include <cuda_runtime.h>
#include <stdint.h>

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
// kRecords (persistent only): also append a compact record per hit.
template <bool kPersistent, int kMinBlocks, bool kRecords = false>
__global__ void __launch_bounds__(kMinBlocks > 0 ? 256 : 1024, kMinBlocks > 0 ? kMinBlocks : 1)
k_propagate(IceDev I, GeomDev G, WorkDev W, RunDev R, uint64_t n_plain) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tables T = stage_tables(smem, I, G);
  __syncthreads();
  const uint64_t total = __ldg(W.meta + 0);
  const uint32_t k = (uint32_t)__ldg(W.meta + 1);
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
    if (W.stats) {
      unsigned long long v0 = steps, v1 = crossings, v2 = births, v3 = slow;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(kFull, v0, o);
        v1 += __shfl_down_sync(kFull, v1, o);
        v2 += __shfl_down_sync(kFull, v2, o);
        v3 += __shfl_down_sync(kFull, v3, o);
      }
      if (lane == 0) {
        atomicAdd(W.stats + 0, v0);
        atomicAdd(W.stats + 1, v1);
        atomicAdd(W.stats + 2, v2);
        atomicAdd(W.stats + 3, v3);
      }
    }
  }
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
  const size_t b = (size_t)ice.L * 16 + (size_t)geom.n_str * 24 + (size_t)geom.nx * geom.ny;
  return (b + 15) & ~(size_t)15;
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

cudaError_t set_propagate_smem_limit(size_t smem) {
  const void* fns[] = {(const void*)k_propagate<true, 0>, (const void*)k_propagate<true, 5>,
                       (const void*)k_propagate<true, 6>, (const void*)k_propagate<false, 0>,
                       (const void*)k_propagate<true, 0, true>};
  cudaError_t e;
  for (const void* f : fns) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_first_hit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t propagate_occupancy(int block_threads, size_t smem, int variant, int* blocks_per_sm) {
  if (variant == 5)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate<true, 5>, 256,
                                                         smem);
  if (variant == 6)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate<true, 6>, 256,
                                                         smem);
  if (variant == kVariantRecords)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, k_propagate<true, 0, true>, block_threads, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_propagate<true, 0>,
                                                       block_threads, smem);
}

cudaError_t launch_propagate(bool persistent, const IceDev& ice, const GeomDev& geom,
                             const WorkDev& work, const RunDev& run, int block_threads,
                             int grid_blocks, uint64_t n_photons_host, size_t smem,
                             cudaStream_t st, int variant) {
  if (persistent) {
    if (variant == 5)
      k_propagate<true, 5><<<grid_blocks, 256, smem, st>>>(ice, geom, work, run, 0);
    else if (variant == 6)
      k_propagate<true, 6><<<grid_blocks, 256, smem, st>>>(ice, geom, work, run, 0);
    else if (variant == kVariantRecords)
      k_propagate<true, 0, true><<<grid_blocks, block_threads, smem, st>>>(ice, geom, work, run, 0);
    else
      k_propagate<true, 0><<<grid_blocks, block_threads, smem, st>>>(ice, geom, work, run, 0);
  } else {
    if (n_photons_host == 0) return cudaSuccess;
    const uint64_t nb = (n_photons_host + block_threads - 1) / block_threads;
    k_propagate<false, 0><<<(unsigned)nb, block_threads, smem, st>>>(ice, geom, work, run,
                                                                      n_photons_host);
  }
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
