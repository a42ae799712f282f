// C ABI of the photon propagator (declared in include/pp.h): context,
// geometry and ice loading (with the host-side preprocessing of the hit-test
// tables), argument checking, staging of host buffers, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pp.h"
#include "pp_internal.h"
#include "pp_nvtx.h"
#include "mlp_internal.h"

using namespace ppk;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

struct pp_ctx {
  pp_config cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;  // host path: uploads and downloads beside the kernels
  cudaStream_t stream2 = nullptr;      // host path: every other chunk's kernels (tails overlap)
  bool own_stream = false;
  int sm_count = 0;
  std::mutex mu;
  std::string last_error = "no error";

  bool geom_loaded = false, ice_loaded = false;
  GeomDev geom{};
  IceDev ice{};
  // device tables
  DevBuf dom, str, str_range, sdom_z, sdom_idx, clear, cell_off, cell_list, layers;
  // scratch
  DevBuf off, chunk, aux, bsum, meta, work, err, stats;
  // a second set of the expansion's scratch, for chunks launched on stream2
  DevBuf off2, chunk2, aux2, bsum2, meta2, work2;
  // staging for host entry points
  DevBuf s_src, s_begin, s_ids, s_hits, s_counts, s_misc1, s_misc2, s_misc3, s_misc4, s_bad;

  int n_accept = 0;                    // hit-record acceptance polynomial
  float accept[PP_MAX_ACCEPT_COEFFS] = {};

  // defaults: the fastest setting measured on the full-detector batch
  // (1024-thread blocks, one per SM; reserved photons handed out once two
  // lanes are idle)
  int block_threads = 1024;
  int blocks_per_sm = 0;  // 0: occupancy maximum
  int refill = 2;
  int lane_photons = 2;   // 2: the persistent kernel keeps a per-warp photon reserve

  // CUDA graphs of the batched path, keyed by everything a capture bakes in
  struct GraphEntry {
    uint64_t key[12];
    cudaGraphExec_t exec;
    int kernels;
  };
  bool graphs = false;
  uint64_t epoch = 0;
  std::atomic<int> servers{0};  // attached serving loops  // bumped when a device buffer or table the kernels read moves
  std::vector<GraphEntry> graph_cache;

  // benchmark timing of propagation launches
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> event_pool;
  uint64_t kernels_launched = 0;
  // device memory the context holds (its DevBufs) and its cudaMalloc calls
  uint64_t device_bytes = 0, n_allocations = 0;
};

namespace {

int fail(pp_ctx* c, int code, const std::string& msg) {
  if (c) c->last_error = msg;
  return code;
}

int cuda_fail(pp_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int fail_ctx(pp_ctx* c, int code, const char* msg) { return fail(c, code, msg); }
int cuda_fail_ctx(pp_ctx* c, cudaError_t e, const char* where) { return cuda_fail(c, e, where); }

#define PP_CUDA(expr)                                   \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)

int ensure(pp_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return PP_OK;
  ctx->epoch += 1;  // captured graphs hold the old address
  // the old buffer may still be read by queued work on the context's streams
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && ctx->stream2) e = cudaStreamSynchronize(ctx->stream2);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  if (b.p) cudaFree(b.p);
  ctx->device_bytes -= b.cap;
  b.p = nullptr;
  b.cap = 0;
  size_t nb = std::max<size_t>(bytes, 256);
  nb = (nb + 255) & ~(size_t)255;
  ctx->n_allocations += 1;
  e = cudaMalloc(&b.p, nb);
  if (e != cudaSuccess) {
    b.p = nullptr;
    (void)cudaGetLastError();
    return fail(ctx, PP_ENOMEM, std::string("cudaMalloc of ") + std::to_string(nb) +
                                     " bytes failed: " + cudaGetErrorString(e));
  }
  b.cap = nb;
  ctx->device_bytes += nb;
  return PP_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

template <class T>
int upload(pp_ctx* ctx, DevBuf& b, const std::vector<T>& v) {
  int rc = ensure(ctx, b, v.size() * sizeof(T));
  if (rc) return rc;
  if (!v.empty()) PP_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PP_OK;
}

cudaStream_t pick_stream(pp_ctx* ctx, void* s) {
  return s ? static_cast<cudaStream_t>(s) : ctx->stream;
}

bool source_ok(const pp_source& s) {
  return std::isfinite(s.x) && std::isfinite(s.y) && std::isfinite(s.z) && std::isfinite(s.dx) &&
         std::isfinite(s.dy) && std::isfinite(s.dz) && std::isfinite(s.length) && s.length >= 0.f &&
         (s.dx != 0.f || s.dy != 0.f || s.dz != 0.f) && s.type <= PP_SRC_CASCADE;
}

int check_sources(pp_ctx* ctx, const pp_source* src, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!source_ok(src[i]))
      return fail(ctx, PP_EINVAL, "source " + std::to_string(i) +
                                      " has a non-finite field, a zero direction, a negative "
                                      "length or an unknown type");
  return PP_OK;
}

// The same check on sources already copied to the device (one kernel and a
// 8-byte read-back instead of a host loop over every source).
int check_sources_device(pp_ctx* ctx, const pp_source* d_src, int64_t n, cudaStream_t st) {
  if (n <= 0) return PP_OK;
  int rc;
  if ((rc = ensure(ctx, ctx->s_bad, sizeof(unsigned long long)))) return rc;
  auto* bad = static_cast<unsigned long long*>(ctx->s_bad.p);
  PP_CUDA(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), st));
  PP_CUDA(launch_check_sources(d_src, n, 0, bad, st));
  unsigned long long first = 0;
  PP_CUDA(cudaMemcpyAsync(&first, bad, sizeof(first), cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaStreamSynchronize(st));
  if (first != ~0ull)
    return fail(ctx, PP_EINVAL, "source " + std::to_string(first) +
                                    " has a non-finite field, a zero direction, a negative "
                                    "length or an unknown type");
  return PP_OK;
}

int check_loaded(pp_ctx* ctx) {
  if (!ctx->geom_loaded || !ctx->ice_loaded)
    return fail(ctx, PP_ENOTLOADED, "load geometry and ice before propagating");
  return PP_OK;
}

// Register-capped kernel variant for the launch settings (see launch_propagate),
// with the photon reserve when two photons per lane are asked for.
// One photon per lane: 256-thread blocks at 5 or 6 per SM use kernels capped at
// 48 / 40 registers.  Two photons per lane: 256-thread blocks at 3 per SM use
// a kernel allowed 80 registers (the reserve's birth pass holds a second
// photon's state beside the lane's own).
int kernel_variant(const pp_ctx* ctx, bool records = false) {
  const bool reserve = ctx->lane_photons == 2;
  int v = 0;
  if (records) v = kVariantRecords;
  else if (ctx->block_threads == 256 && !reserve &&
           (ctx->blocks_per_sm == 5 || ctx->blocks_per_sm == 6))
    v = ctx->blocks_per_sm;
  else if (ctx->block_threads == 256 && reserve && ctx->blocks_per_sm == 3)
    v = 3;
  return reserve ? v + kVariantReserve : v;
}

// Dynamic shared memory of a launch of `variant` (0 for the kernels without a
// reserve): the staged tables, plus the photon reserve of reserve variants;
// raises the kernels' limit when needed.
int prepare_smem(pp_ctx* ctx, size_t* smem, int variant) {
  *smem = tables_smem_bytes(ctx->ice, ctx->geom);
  if (variant >= kVariantReserve) {
    const int base = variant - kVariantReserve;
    const int bt = (base == 3 || base == 5 || base == 6) ? 256 : ctx->block_threads;
    *smem += reserve_smem_bytes(bt, base == kVariantRecords);
  }
  // raises the kernels' limit (process-wide, never lowered) when needed
  const cudaError_t e = set_propagate_smem_limit(std::max<size_t>(*smem, 48 * 1024));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
  return PP_OK;
}

int grid_blocks(pp_ctx* ctx, size_t smem, int* out, int variant = -1) {
  int occ = 0;
  cudaError_t e = propagate_occupancy(ctx->block_threads, smem,
                                      variant < 0 ? kernel_variant(ctx) : variant, &occ);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ < 1) return fail(ctx, PP_EINVAL, "propagation kernel does not fit on an SM");
  const int bps = ctx->blocks_per_sm > 0 ? std::min(ctx->blocks_per_sm, occ) : occ;
  *out = bps * ctx->sm_count;
  return PP_OK;
}

RunDev run_params(const pp_ctx* ctx) {
  RunDev r;
  for (uint32_t i = 0; i < 10; ++i) {
    r.key_x[i] = (uint32_t)ctx->cfg.seed + 0x9E3779B9u * i;
    r.key_y[i] = (uint32_t)(ctx->cfg.seed >> 32) + 0xBB67AE85u * i;
  }
  r.max_steps = ctx->cfg.max_steps;
  r.cos_cherenkov = (float)std::cos(41.0 * 3.14159265358979323846 / 180.0);
  r.sin_cherenkov = (float)std::sin(41.0 * 3.14159265358979323846 / 180.0);
  r.refill = ctx->refill;
  r.ns_per_m_emit = (float)(1.0 / kLightSpeedMperNs);
  r.ns_per_m_path = (float)(kGroupIndexDefault / kLightSpeedMperNs);
  r.n_accept = ctx->n_accept;
  for (int i = 0; i < PP_MAX_ACCEPT_COEFFS; ++i) r.accept[i] = ctx->accept[i];
  return r;
}

int ensure_scratch(pp_ctx* ctx, int64_t n_src, bool with_events) {
  int rc;
  if ((rc = ensure(ctx, ctx->off, sizeof(uint64_t) * (size_t)(n_src + 1)))) return rc;
  if ((rc = ensure(ctx, ctx->chunk, sizeof(uint32_t) * (size_t)(n_src + 2)))) return rc;
  if (with_events && (rc = ensure(ctx, ctx->aux, sizeof(SrcAux) * (size_t)std::max<int64_t>(n_src, 1))))
    return rc;
  const int64_t nb = (n_src + kScanTile - 1) / kScanTile;
  if ((rc = ensure(ctx, ctx->bsum, sizeof(uint64_t) * (size_t)std::max<int64_t>(nb, 1)))) return rc;
  if ((rc = ensure(ctx, ctx->meta, sizeof(uint64_t) * 2))) return rc;
  if ((rc = ensure(ctx, ctx->work, sizeof(uint64_t)))) return rc;
  return PP_OK;
}

ExpandBufs expand_bufs(pp_ctx* ctx, bool with_events) {
  ExpandBufs b;
  b.off = static_cast<uint64_t*>(ctx->off.p);
  b.chunk_src = static_cast<uint32_t*>(ctx->chunk.p);
  b.aux = with_events ? static_cast<SrcAux*>(ctx->aux.p) : nullptr;
  b.bsum = static_cast<uint64_t*>(ctx->bsum.p);
  b.meta = static_cast<uint64_t*>(ctx->meta.p);
  return b;
}

WorkDev work_desc(pp_ctx* ctx, const pp_source* d_src, int64_t n_src, bool with_events,
                  const int64_t* d_begin, const uint64_t* d_ids, uint64_t* d_hits,
                  uint64_t* d_counts, uint32_t single_ev_lo) {
  WorkDev w;
  w.src = d_src;
  w.off = static_cast<const uint64_t*>(ctx->off.p);
  w.chunk_src = static_cast<const uint32_t*>(ctx->chunk.p);
  w.aux = with_events ? static_cast<const SrcAux*>(ctx->aux.p) : nullptr;
  (void)d_begin;
  (void)d_ids;
  w.meta = static_cast<const uint64_t*>(ctx->meta.p);
  w.work = static_cast<unsigned long long*>(ctx->work.p);
  w.hits = reinterpret_cast<unsigned long long*>(d_hits);
  w.counts = reinterpret_cast<unsigned long long*>(d_counts);
  w.err = static_cast<int*>(ctx->err.p);
  w.stats = static_cast<unsigned long long*>(ctx->stats.p);
  w.n_src = (int)n_src;
  w.single_event_lo = single_ev_lo;
  w.g_begin = 0;
  w.g_end = ~0ull;
  w.records = nullptr;
  w.n_records = nullptr;
  w.max_records = 0;
  return w;
}

int take_event(pp_ctx* ctx, cudaEvent_t* ev) {
  if (!ctx->event_pool.empty()) {
    *ev = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return PP_OK;
  }
  PP_CUDA(cudaEventCreate(ev));
  return PP_OK;
}

// Launches the propagation kernel, bracketed by timing events when enabled.
int timed_propagate(pp_ctx* ctx, bool persistent, const WorkDev& w, const RunDev& run, int grid,
                    uint64_t n_photons, size_t smem, cudaStream_t st, int variant = -1) {
  NvtxRange range("pp.propagate");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc;
  if (ctx->timing) {
    if ((rc = take_event(ctx, &e0)) || (rc = take_event(ctx, &e1))) return rc;
    PP_CUDA(cudaEventRecord(e0, st));
  }
  if (variant < 0) variant = persistent ? kernel_variant(ctx) : 0;
  // the plain path (one thread per photon, one launch per event) keeps its
  // own block size: the persistent kernel's 1024-thread blocks leave long
  // tails of idle threads there
  PP_CUDA(launch_propagate(persistent, ctx->ice, ctx->geom, w, run,
                           persistent ? ctx->block_threads : kPlainThreads, grid, n_photons, smem,
                           st, variant));
  ctx->kernels_launched += 1;
  if (ctx->timing) {
    PP_CUDA(cudaEventRecord(e1, st));
    ctx->pending.emplace_back(e0, e1);
  }
  return PP_OK;
}

int expand(pp_ctx* ctx, const pp_source* d_src, int64_t n_src, const int64_t* d_begin,
           const uint64_t* d_ids, int n_events, bool with_events, cudaStream_t st) {
  NvtxRange range("pp.expand");
  PP_CUDA(launch_expand(d_src, n_src, d_begin, d_ids, n_events, expand_bufs(ctx, with_events), st));
  ctx->kernels_launched += (n_src <= kSmallMax) ? 1 : 4;
  return PP_OK;
}

// Compact hit records requested from the batched path.
struct RecordsOut {
  pp_hit* records;
  uint64_t capacity;
  uint64_t* count;     // device: total hits (zeroed by the call)
  float group_index;
};

// Batched persistent path on device data (the lock is held by the caller).
int batch_async(pp_ctx* ctx, int32_t n_events, const uint64_t* d_ids, const int64_t* d_begin,
                const pp_source* d_src, int64_t n_src, uint64_t* d_hits, uint64_t* d_counts,
                cudaStream_t st, const RecordsOut* rec = nullptr) {
  NvtxRange range("pp.batch");
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  if (n_events < 0 || n_src < 0 || n_src > kMaxSources)
    return fail(ctx, PP_EINVAL, "n_events/n_src out of range (n_src <= 33554432 per call)");
  if (n_events == 0) return PP_OK;
  if (!d_ids || !d_begin || !d_hits || !d_counts || (n_src > 0 && !d_src))
    return fail(ctx, PP_EINVAL, "null device pointer");
  if (rec && (!rec->count || (rec->capacity > 0 && !rec->records) || n_src > 0xffffffffll ||
              !(rec->group_index >= 1.0f && rec->group_index < 10.0f)))
    return fail(ctx, PP_EINVAL, "hit records: need a count pointer, a buffer for capacity > 0 "
                                "and 1 <= group_index < 10");
  const size_t hb = sizeof(uint64_t) * (size_t)n_events * ctx->geom.n_dom;
  const int variant = kernel_variant(ctx, rec != nullptr);
  size_t smem = 0;
  int grid = 0;
  if (n_src > 0) {
    if ((rc = ensure_scratch(ctx, n_src, true))) return rc;
    if ((rc = prepare_smem(ctx, &smem, variant))) return rc;
    if ((rc = grid_blocks(ctx, smem, &grid, variant))) return rc;
  }
  auto enqueue = [&]() -> int {
    if (hb) PP_CUDA(cudaMemsetAsync(d_hits, 0, hb, st));
    PP_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 4 * (size_t)n_events, st));
    if (rec) PP_CUDA(cudaMemsetAsync(rec->count, 0, sizeof(uint64_t), st));
    if (n_src == 0) return PP_OK;
    PP_CUDA(cudaMemsetAsync(ctx->work.p, 0, sizeof(uint64_t), st));
    int r;
    if ((r = expand(ctx, d_src, n_src, d_begin, d_ids, n_events, true, st))) return r;
    WorkDev w = work_desc(ctx, d_src, n_src, true, d_begin, d_ids, d_hits, d_counts, 0);
    RunDev run = run_params(ctx);
    if (rec) {
      w.records = rec->records;
      w.n_records = reinterpret_cast<unsigned long long*>(rec->count);
      w.max_records = rec->capacity;
      run.ns_per_m_path = (float)(rec->group_index / kLightSpeedMperNs);
    }
    return timed_propagate(ctx, true, w, run, grid, 0, smem, st, variant);
  };
  if (!ctx->graphs || ctx->timing || st == nullptr || rec) return enqueue();
  // CUDA graph: capture this exact launch sequence once, replay it afterwards
  const uint64_t key[12] = {(uint64_t)n_events, (uint64_t)n_src, (uint64_t)d_ids, (uint64_t)d_begin,
                            (uint64_t)d_src, (uint64_t)d_hits, (uint64_t)d_counts, (uint64_t)st,
                            ctx->epoch, (uint64_t)ctx->block_threads,
                            (uint64_t)ctx->blocks_per_sm,
                            (uint64_t)ctx->refill | (uint64_t)ctx->lane_photons << 32};
  for (const auto& g : ctx->graph_cache) {
    if (std::memcmp(g.key, key, sizeof(key)) == 0) {
      PP_CUDA(cudaGraphLaunch(g.exec, st));
      ctx->kernels_launched += g.kernels;
      return PP_OK;
    }
  }
  PP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const uint64_t k0 = ctx->kernels_launched;
  rc = enqueue();
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (rc || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc ? rc : cuda_fail(ctx, ec, "cudaStreamEndCapture");
  }
  pp_ctx::GraphEntry g;
  std::memcpy(g.key, key, sizeof(key));
  g.kernels = (int)(ctx->kernels_launched - k0);
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ctx, ei, "cudaGraphInstantiate");
  if (ctx->graph_cache.size() >= 8) {
    cudaGraphExecDestroy(ctx->graph_cache.front().exec);
    ctx->graph_cache.erase(ctx->graph_cache.begin());
  }
  ctx->graph_cache.push_back(g);
  PP_CUDA(cudaGraphLaunch(g.exec, st));  // the capture only recorded the work
  return PP_OK;
}

// Photons [g0, g1) of one event through the persistent kernel, optionally
// adding to the outputs (the lock is held by the caller).
int range_async(pp_ctx* ctx, uint64_t event_id, const pp_source* d_src, int64_t n_src,
                uint64_t g0, uint64_t g1, bool accumulate, uint64_t* d_hits, uint64_t* d_counts,
                cudaStream_t st) {
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  if (n_src < 0 || n_src > kMaxSources || g1 < g0)
    return fail(ctx, PP_EINVAL, "need 0 <= n_src <= 33554432 and photon_begin <= photon_end");
  if (!d_hits || !d_counts || (n_src > 0 && !d_src)) return fail(ctx, PP_EINVAL, "null pointer");
  if (!accumulate) {
    if (ctx->geom.n_dom)
      PP_CUDA(cudaMemsetAsync(d_hits, 0, sizeof(uint64_t) * (size_t)ctx->geom.n_dom, st));
    PP_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 4, st));
  }
  if (n_src == 0 || g1 == g0) return PP_OK;
  if ((rc = ensure_scratch(ctx, n_src, false))) return rc;
  size_t smem;
  if ((rc = prepare_smem(ctx, &smem, kernel_variant(ctx)))) return rc;
  int grid;
  if ((rc = grid_blocks(ctx, smem, &grid))) return rc;
  PP_CUDA(cudaMemsetAsync(ctx->work.p, 0, sizeof(uint64_t), st));
  if ((rc = expand(ctx, d_src, n_src, nullptr, nullptr, 1, false, st))) return rc;
  WorkDev w = work_desc(ctx, d_src, n_src, false, nullptr, nullptr, d_hits, d_counts,
                        (uint32_t)event_id);
  w.g_begin = g0;
  w.g_end = g1;
  return timed_propagate(ctx, true, w, run_params(ctx), grid, 0, smem, st);
}

// Plain path: per event, expansion and one thread per photon.
int plain_async(pp_ctx* ctx, int32_t n_events, const uint64_t* h_ids, const int64_t* h_begin,
                const uint64_t* h_photons, const pp_source* d_src, uint64_t* d_hits,
                uint64_t* d_counts, cudaStream_t st) {
  NvtxRange range("pp.plain");
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  if (n_events < 0) return fail(ctx, PP_EINVAL, "n_events < 0");
  if (n_events == 0) return PP_OK;
  if (!h_ids || !h_begin || !h_photons || !d_hits || !d_counts)
    return fail(ctx, PP_EINVAL, "null pointer");
  int64_t max_src = 0;
  for (int32_t e = 0; e < n_events; ++e) {
    const int64_t n = h_begin[e + 1] - h_begin[e];
    if (n < 0 || h_begin[0] != 0) return fail(ctx, PP_EINVAL, "src_begin must start at 0 and not decrease");
    max_src = std::max(max_src, n);
  }
  if (max_src > kMaxSources) return fail(ctx, PP_EINVAL, "too many sources in one event");
  if (max_src > 0 && !d_src) return fail(ctx, PP_EINVAL, "null source pointer");
  const int n_dom = ctx->geom.n_dom;
  if (n_dom) PP_CUDA(cudaMemsetAsync(d_hits, 0, sizeof(uint64_t) * (size_t)n_events * n_dom, st));
  PP_CUDA(cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 4 * (size_t)n_events, st));
  if ((rc = ensure_scratch(ctx, std::max<int64_t>(max_src, 1), false))) return rc;
  size_t smem;
  if ((rc = prepare_smem(ctx, &smem, 0))) return rc;
  const RunDev run = run_params(ctx);
  for (int32_t e = 0; e < n_events; ++e) {
    const int64_t n = h_begin[e + 1] - h_begin[e];
    if (n == 0 || h_photons[e] == 0) continue;
    const pp_source* s = d_src + h_begin[e];
    if ((rc = expand(ctx, s, n, nullptr, nullptr, 1, false, st))) return rc;
    const WorkDev w = work_desc(ctx, s, n, false, nullptr, nullptr, d_hits + (size_t)e * n_dom,
                                d_counts + 4 * (size_t)e, (uint32_t)h_ids[e]);
    if ((rc = timed_propagate(ctx, false, w, run, 0, h_photons[e], smem, st))) return rc;
  }
  return PP_OK;
}

void drop_graphs(pp_ctx* ctx) {
  for (auto& g : ctx->graph_cache) cudaGraphExecDestroy(g.exec);
  ctx->graph_cache.clear();
  ctx->epoch += 1;
}

int sync_and_check(pp_ctx* ctx, cudaStream_t st) {
  PP_CUDA(cudaStreamSynchronize(st));
  int flag = 0;
  PP_CUDA(cudaMemcpy(&flag, ctx->err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    PP_CUDA(cudaMemset(ctx->err.p, 0, sizeof(int)));
    return fail(ctx, PP_EDEVICE, "device error flag " + std::to_string(flag) +
                                     " (malformed source seen by a kernel)");
  }
  return PP_OK;
}

// Host batch, batched path, large inputs: the events are cut into 3 chunks
// (10 %, 80 %, 10 % of the sources); a copy stream uploads every chunk and
// downloads each chunk's results once its propagation (on the context's
// stream) is done, so transfers overlap the kernels.  The sources are
// checked on the device; a malformed one fails the call with PP_EINVAL after
// the work (the kernels skip malformed sources).
// Exchanges the expansion scratch the launch helpers use with the second set.
void swap_scratch(pp_ctx* ctx) {
  std::swap(ctx->off, ctx->off2);
  std::swap(ctx->chunk, ctx->chunk2);
  std::swap(ctx->aux, ctx->aux2);
  std::swap(ctx->bsum, ctx->bsum2);
  std::swap(ctx->meta, ctx->meta2);
  std::swap(ctx->work, ctx->work2);
}

int batch_host_pipelined(pp_ctx* ctx, int32_t n_events, const uint64_t* ids, const int64_t* begin,
                         const pp_source* src, uint64_t* hits, uint64_t* counts) {
  NvtxRange range("pp.host_pipeline");
  int rc;
  const int64_t n_src = begin[n_events];
  const int n_dom = ctx->geom.n_dom;
  cudaStream_t st = ctx->stream;
  if (!ctx->copy_stream) PP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  if (!ctx->stream2) PP_CUDA(cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
  cudaStream_t cs = ctx->copy_stream;
  // chunks alternate between the two compute streams, each with its own
  // expansion scratch, so that a chunk's kernels start while the previous
  // chunk's last photons finish; a chunk waits only for its own upload and
  // (same stream) for the chunk two before it, which used the same scratch
  cudaStream_t cst[2] = {st, ctx->stream2};
  // chunks: event ranges cut at 10 % and 90 % of the sources
  std::vector<int32_t> cut{0};
  // a small first chunk (its upload is exposed), a small last one (its
  // download is exposed), the bulk in between
  static constexpr double edges[] = {0.1, 0.9};
  for (double edge : edges) {
    const int64_t target = (int64_t)(edge * (double)n_src);
    int32_t e = cut.back();
    while (e < n_events && begin[e] < target) ++e;
    if (e > cut.back() && e < n_events) cut.push_back(e);
  }
  cut.push_back(n_events);
  const int nc = (int)cut.size() - 1;
  if ((rc = ensure(ctx, ctx->s_src, sizeof(pp_source) * (size_t)std::max<int64_t>(n_src, 1)))) return rc;
  if ((rc = ensure(ctx, ctx->s_begin, sizeof(int64_t) * (size_t)(n_events + nc)))) return rc;
  if ((rc = ensure(ctx, ctx->s_ids, sizeof(uint64_t) * (size_t)n_events))) return rc;
  if ((rc = ensure(ctx, ctx->s_hits, sizeof(uint64_t) * (size_t)n_events * std::max(n_dom, 1)))) return rc;
  if ((rc = ensure(ctx, ctx->s_counts, sizeof(uint64_t) * 4 * (size_t)n_events))) return rc;
  if ((rc = ensure(ctx, ctx->s_bad, sizeof(unsigned long long)))) return rc;
  auto* bad = static_cast<unsigned long long*>(ctx->s_bad.p);
  auto* d_src = static_cast<pp_source*>(ctx->s_src.p);
  auto* d_begin = static_cast<int64_t*>(ctx->s_begin.p);
  auto* d_ids = static_cast<uint64_t*>(ctx->s_ids.p);
  auto* d_hits = static_cast<uint64_t*>(ctx->s_hits.p);
  auto* d_counts = static_cast<uint64_t*>(ctx->s_counts.p);
  // each chunk's source offsets relative to its first source (kept until the end)
  std::vector<int64_t> rel((size_t)(n_events + nc));
  std::vector<cudaEvent_t> up(nc, nullptr), done(nc, nullptr);
  cudaEvent_t cleared = nullptr;
  const bool keep_graphs = ctx->graphs;
  ctx->graphs = false;  // captured graphs are keyed without the scratch set
  auto release = [&]() {
    for (auto& e : up) if (e) cudaEventDestroy(e);
    for (auto& e : done) if (e) cudaEventDestroy(e);
    if (cleared) cudaEventDestroy(cleared);
    ctx->graphs = keep_graphs;
  };
  auto step = [&]() -> int {
    PP_CUDA(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), st));
    PP_CUDA(cudaEventCreateWithFlags(&cleared, cudaEventDisableTiming));
    PP_CUDA(cudaEventRecord(cleared, st));
    PP_CUDA(cudaStreamWaitEvent(ctx->stream2, cleared, 0));
    for (int k = 0; k < nc; ++k) {
      const int32_t e0 = cut[k], e1 = cut[k + 1];
      const int64_t s0 = begin[e0], s1 = begin[e1];
      int64_t* rk = rel.data() + e0 + k;
      for (int32_t e = e0; e <= e1; ++e) rk[e - e0] = begin[e] - s0;
      PP_CUDA(cudaEventCreateWithFlags(&up[k], cudaEventDisableTiming));
      PP_CUDA(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming));
      if (s1 > s0)
        PP_CUDA(cudaMemcpyAsync(d_src + s0, src + s0, sizeof(pp_source) * (size_t)(s1 - s0),
                                cudaMemcpyHostToDevice, cs));
      PP_CUDA(cudaMemcpyAsync(d_begin + e0 + k, rk, sizeof(int64_t) * (size_t)(e1 - e0 + 1),
                              cudaMemcpyHostToDevice, cs));
      PP_CUDA(cudaMemcpyAsync(d_ids + e0, ids + e0, sizeof(uint64_t) * (size_t)(e1 - e0),
                              cudaMemcpyHostToDevice, cs));
      PP_CUDA(cudaEventRecord(up[k], cs));
    }
    for (int k = 0; k < nc; ++k) {
      const int32_t e0 = cut[k], e1 = cut[k + 1];
      const int64_t s0 = begin[e0], s1 = begin[e1];
      cudaStream_t ks = cst[k & 1];
      PP_CUDA(cudaStreamWaitEvent(ks, up[k], 0));
      PP_CUDA(launch_check_sources(d_src + s0, s1 - s0, s0, bad, ks));
      if (k & 1) swap_scratch(ctx);
      int r = batch_async(ctx, e1 - e0, d_ids + e0, d_begin + e0 + k, d_src + s0, s1 - s0,
                          d_hits + (size_t)e0 * n_dom, d_counts + (size_t)e0 * 4, ks);
      if (k & 1) swap_scratch(ctx);
      if (r) return r;
      PP_CUDA(cudaEventRecord(done[k], ks));
      PP_CUDA(cudaStreamWaitEvent(cs, done[k], 0));
      if (n_dom)
        PP_CUDA(cudaMemcpyAsync(hits + (size_t)e0 * n_dom, d_hits + (size_t)e0 * n_dom,
                                sizeof(uint64_t) * (size_t)(e1 - e0) * n_dom,
                                cudaMemcpyDeviceToHost, cs));
      PP_CUDA(cudaMemcpyAsync(counts + (size_t)e0 * 4, d_counts + (size_t)e0 * 4,
                              sizeof(uint64_t) * 4 * (size_t)(e1 - e0), cudaMemcpyDeviceToHost, cs));
    }
    PP_CUDA(cudaStreamSynchronize(cs));
    return PP_OK;
  };
  rc = step();
  release();
  if (rc) {
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(ctx->stream2);
    cudaStreamSynchronize(st);
    return rc;
  }
  PP_CUDA(cudaStreamSynchronize(ctx->stream2));
  unsigned long long first = 0;
  PP_CUDA(cudaMemcpy(&first, bad, sizeof(first), cudaMemcpyDeviceToHost));
  if (first != ~0ull) {
    PP_CUDA(cudaStreamSynchronize(st));
    PP_CUDA(cudaMemset(ctx->err.p, 0, sizeof(int)));  // the kernels' flag for the same sources
    return fail(ctx, PP_EINVAL, "source " + std::to_string(first) +
                                    " has a non-finite field, a zero direction, a negative "
                                    "length or an unknown type");
  }
  return sync_and_check(ctx, st);
}

// Host batch: stage inputs, run the given path, copy results back.
int batch_host(pp_ctx* ctx, bool plain, int32_t n_events, const uint64_t* ids,
               const int64_t* begin, const pp_source* src, uint64_t* hits, uint64_t* counts) {
  NvtxRange range("pp.host_batch");
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  if (n_events < 0 || (n_events > 0 && (!ids || !begin || !hits || !counts)))
    return fail(ctx, PP_EINVAL, "null pointer or negative n_events");
  if (n_events == 0) return PP_OK;
  if (begin[0] != 0) return fail(ctx, PP_EINVAL, "src_begin[0] must be 0");
  for (int32_t e = 0; e < n_events; ++e)
    if (begin[e + 1] < begin[e]) return fail(ctx, PP_EINVAL, "src_begin decreases");
  const int64_t n_src = begin[n_events];
  if (n_src > 0 && !src) return fail(ctx, PP_EINVAL, "null source pointer");
  if (n_src > kMaxSources) return fail(ctx, PP_EINVAL, "more than 33554432 sources per call");
  if (!plain && n_src >= (1 << 18) && n_events >= 4)
    return batch_host_pipelined(ctx, n_events, ids, begin, src, hits, counts);
  const int n_dom = ctx->geom.n_dom;
  cudaStream_t st = ctx->stream;
  if ((rc = ensure(ctx, ctx->s_src, sizeof(pp_source) * (size_t)std::max<int64_t>(n_src, 1)))) return rc;
  if ((rc = ensure(ctx, ctx->s_begin, sizeof(int64_t) * (size_t)(n_events + 1)))) return rc;
  if ((rc = ensure(ctx, ctx->s_ids, sizeof(uint64_t) * (size_t)n_events))) return rc;
  if ((rc = ensure(ctx, ctx->s_hits, sizeof(uint64_t) * (size_t)n_events * std::max(n_dom, 1)))) return rc;
  if ((rc = ensure(ctx, ctx->s_counts, sizeof(uint64_t) * 4 * (size_t)n_events))) return rc;
  if (n_src)
    PP_CUDA(cudaMemcpyAsync(ctx->s_src.p, src, sizeof(pp_source) * n_src, cudaMemcpyHostToDevice, st));
  PP_CUDA(cudaMemcpyAsync(ctx->s_begin.p, begin, sizeof(int64_t) * (n_events + 1), cudaMemcpyHostToDevice, st));
  PP_CUDA(cudaMemcpyAsync(ctx->s_ids.p, ids, sizeof(uint64_t) * n_events, cudaMemcpyHostToDevice, st));
  uint64_t* d_hits = static_cast<uint64_t*>(ctx->s_hits.p);
  uint64_t* d_counts = static_cast<uint64_t*>(ctx->s_counts.p);
  const pp_source* d_src = static_cast<const pp_source*>(ctx->s_src.p);
  if ((rc = check_sources_device(ctx, d_src, n_src, st))) return rc;
  if (plain) {
    std::vector<uint64_t> ph(n_events, 0);
    for (int32_t e = 0; e < n_events; ++e)
      for (int64_t s = begin[e]; s < begin[e + 1]; ++s) ph[e] += src[s].n_photons;
    rc = plain_async(ctx, n_events, ids, begin, ph.data(), d_src, d_hits, d_counts, st);
  } else {
    rc = batch_async(ctx, n_events, static_cast<const uint64_t*>(ctx->s_ids.p),
                     static_cast<const int64_t*>(ctx->s_begin.p), d_src, n_src, d_hits, d_counts, st);
  }
  if (rc) return rc;
  if (n_dom)
    PP_CUDA(cudaMemcpyAsync(hits, d_hits, sizeof(uint64_t) * (size_t)n_events * n_dom, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaMemcpyAsync(counts, d_counts, sizeof(uint64_t) * 4 * (size_t)n_events, cudaMemcpyDeviceToHost, st));
  return sync_and_check(ctx, st);
}

}  // namespace

namespace ppk {

int LaunchView::fail(int code, const char* msg) const { return fail_ctx(ctx, code, msg); }

int LaunchView::cuda_fail(cudaError_t e, const char* where) const {
  return cuda_fail_ctx(ctx, e, where);
}

void attach_server(pp_ctx* ctx, int delta) { ctx->servers += delta; }

void count_launches(pp_ctx* ctx, int n) { ctx->kernels_launched += (uint64_t)n; }

int with_launch_view(pp_ctx* ctx, const std::function<int(const LaunchView&)>& fn) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  LaunchView v;
  v.ctx = ctx;
  v.device = ctx->cfg.device;
  v.stream = ctx->stream;
  v.ice = ctx->ice;
  v.geom = ctx->geom;
  v.run = run_params(ctx);
  v.block_threads = ctx->block_threads;
  v.variant = kernel_variant(ctx);
  v.scatter_effective = ctx->cfg.scatter_coeff_is_effective;
  if ((rc = prepare_smem(ctx, &v.smem, v.variant))) return rc;
  if ((rc = grid_blocks(ctx, v.smem, &v.grid_blocks))) return rc;
  v.err = static_cast<int*>(ctx->err.p);
  v.stats = static_cast<unsigned long long*>(ctx->stats.p);
  return fn(v);
}

}  // namespace ppk

extern "C" {

const char* pp_strerror(int code) {
  switch (code) {
    case PP_OK: return "ok";
    case PP_EINVAL: return "invalid argument";
    case PP_ENOTLOADED: return "geometry or ice not loaded";
    case PP_EBUDGET: return "request exceeds the budget";
    case PP_ETIMEDOUT: return "timed out";
    case PP_ECUDA: return "CUDA runtime error";
    case PP_EDEVICE: return "device error flag raised";
    case PP_ENOMEM: return "device allocation failed";
    case PP_ENODEV: return "no usable CUDA device";
    default: return "unknown error";
  }
}

const char* pp_last_error(const pp_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

int pp_config_default(pp_config* cfg) {
  if (!cfg) return PP_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->max_steps = 100000;
  cfg->seed = 0;
  cfg->world_margin_m = 100.0f;
  cfg->depth_of_z0_m = 1950.0f;
  cfg->scatter_coeff_is_effective = 1;
  cfg->stream = nullptr;
  return PP_OK;
}

int pp_create(const pp_config* cfg, pp_ctx** out) {
  if (!cfg || !out) return PP_EINVAL;
  *out = nullptr;
  if (cfg->max_steps == 0 || !(cfg->world_margin_m >= 0.f) || !std::isfinite(cfg->depth_of_z0_m))
    return PP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return PP_ENODEV;
  }
  if (cfg->device < 0 || cfg->device >= ndev) return PP_ENODEV;
  pp_ctx* ctx = new pp_ctx();
  ctx->cfg = *cfg;
  ppk::DeviceScope dev_scope(cfg->device);
  cudaError_t e = dev_scope.status();
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cfg->device);
  if (e == cudaSuccess) {
    if (cfg->stream) {
      ctx->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = (e == cudaSuccess);
    }
  }
  if (e == cudaSuccess) e = ppk::noalloc_setup(cfg->device);
  if (e == cudaSuccess && ensure(ctx, ctx->err, sizeof(int)) == PP_OK &&
      ensure(ctx, ctx->stats, 4 * sizeof(uint64_t)) == PP_OK) {
    e = cudaMemset(ctx->err.p, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->stats.p, 0, 4 * sizeof(uint64_t));
  }
  if (e != cudaSuccess || !ctx->err.p || !ctx->stats.p) {
    (void)cudaGetLastError();
    pp_destroy(ctx);
    return PP_ECUDA;
  }
  *out = ctx;
  return PP_OK;
}

int pp_destroy(pp_ctx* ctx) {
  if (!ctx) return PP_OK;
  ppk::DeviceScope dev_scope(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  DevBuf* bufs[] = {&ctx->dom, &ctx->str, &ctx->str_range, &ctx->sdom_z, &ctx->sdom_idx,
                    &ctx->clear, &ctx->cell_off, &ctx->cell_list, &ctx->layers, &ctx->off,
                    &ctx->chunk, &ctx->aux, &ctx->bsum, &ctx->meta, &ctx->work, &ctx->err,
                    &ctx->stats, &ctx->off2, &ctx->chunk2, &ctx->aux2, &ctx->bsum2, &ctx->meta2,
                    &ctx->work2,
                    &ctx->s_src, &ctx->s_begin, &ctx->s_ids, &ctx->s_hits, &ctx->s_counts,
                    &ctx->s_misc1, &ctx->s_misc2, &ctx->s_misc3, &ctx->s_misc4, &ctx->s_bad};
  drop_graphs(ctx);
  for (DevBuf* b : bufs) release(*b);
  for (auto& pr : ctx->pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
  delete ctx;
  return PP_OK;
}

int pp_load_geometry(pp_ctx* ctx, const float* xyz, const int32_t* string_id, int32_t n_dom,
                     float dom_radius) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->servers > 0) return fail(ctx, PP_EINVAL, "a serving loop is attached to this context");
  if (n_dom < 0 || n_dom > 65535 || (n_dom > 0 && !xyz) || !(dom_radius > 0.f) ||
      !std::isfinite(dom_radius))
    return fail(ctx, PP_EINVAL, "need 0 <= n_dom <= 65535, xyz, dom_radius > 0");
  for (int64_t i = 0; i < 3 * (int64_t)n_dom; ++i)
    if (!std::isfinite(xyz[i])) return fail(ctx, PP_EINVAL, "non-finite DOM coordinate");
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  const double r = dom_radius;
  const double M = ctx->cfg.world_margin_m;
  const double eps = 2e-3;  // slack for FP32 rounding in the culling tests

  // strings: group by id, DOMs by ascending z
  std::map<int32_t, std::vector<int>> groups;
  for (int k = 0; k < n_dom; ++k) groups[string_id ? string_id[k] : 0].push_back(k);
  if ((int)groups.size() > kMaxStrings) return fail(ctx, PP_EINVAL, "more than 4096 strings");
  std::vector<float4> dom(n_dom), str;
  std::vector<int2> rng;
  std::vector<float> sz;
  std::vector<int> sidx;
  std::vector<double> scx, scy, srad;
  double rmax = 0, zmin = 0, zmax = 0;
  for (int k = 0; k < n_dom; ++k) {
    dom[k] = make_float4(xyz[3 * k], xyz[3 * k + 1], xyz[3 * k + 2], 0.f);
    rmax = std::max(rmax, std::hypot((double)xyz[3 * k], (double)xyz[3 * k + 1]));
    if (k == 0 || xyz[3 * k + 2] < zmin) zmin = xyz[3 * k + 2];
    if (k == 0 || xyz[3 * k + 2] > zmax) zmax = xyz[3 * k + 2];
  }
  for (auto& kv : groups) {
    std::vector<int>& ks = kv.second;
    std::sort(ks.begin(), ks.end(), [&](int p, int q) {
      return xyz[3 * p + 2] < xyz[3 * q + 2] || (xyz[3 * p + 2] == xyz[3 * q + 2] && p < q);
    });
    double cx = 0, cy = 0;
    for (int k : ks) {
      cx += xyz[3 * k];
      cy += xyz[3 * k + 1];
    }
    cx /= ks.size();
    cy /= ks.size();
    double rad = 0;
    for (int k : ks) rad = std::max(rad, std::hypot(xyz[3 * k] - cx, xyz[3 * k + 1] - cy));
    rad += r + eps;
    rng.push_back(make_int2((int)sz.size(), (int)ks.size()));
    for (int k : ks) {
      sz.push_back(xyz[3 * k + 2]);
      sidx.push_back(k);
    }
    str.push_back(make_float4((float)cx, (float)cy, (float)rad, 0.f));
    scx.push_back(cx);
    scy.push_back(cy);
    srad.push_back(rad);
  }
  const int n_str = (int)str.size();
  // world cylinder
  const double R = rmax + M, zlo = (n_dom ? zmin : 0.0) - M, zhi = (n_dom ? zmax : 0.0) + M;
  // cell grid over [-R, R]^2: clearance (u8, units of 0.25 m) and string lists
  const int nside = 181;  // nside^2 <= kMaxCells
  const double cell = std::max(2.0 * R / nside, 1.0);
  const int nx = std::max(1, (int)std::ceil(2.0 * R / cell));
  const int ny = nx;
  const double unit = 0.25, halo = cell;
  std::vector<uint8_t> clear((size_t)nx * ny);
  std::vector<uint32_t> coff((size_t)nx * ny + 1, 0);
  std::vector<uint16_t> clist;
  for (int iy = 0; iy < ny; ++iy) {
    for (int ix = 0; ix < nx; ++ix) {
      const double x0 = -R + ix * cell, x1 = x0 + cell, y0 = -R + iy * cell, y1 = y0 + cell;
      double cl = 1e30;
      const size_t c = (size_t)iy * nx + ix;
      coff[c] = (uint32_t)clist.size();
      for (int s = 0; s < n_str; ++s) {
        const double ddx = std::max({x0 - scx[s], 0.0, scx[s] - x1});
        const double ddy = std::max({y0 - scy[s], 0.0, scy[s] - y1});
        const double d = std::hypot(ddx, ddy);
        cl = std::min(cl, d - srad[s]);
        if (d <= srad[s] + halo + eps) clist.push_back((uint16_t)s);
      }
      const double q = std::floor((cl - 0.01) / unit);
      clear[c] = (uint8_t)std::max(0.0, std::min(255.0, q));
    }
  }
  coff[(size_t)nx * ny] = (uint32_t)clist.size();
  if (clist.empty()) clist.push_back(0);
  if (sz.empty()) {
    sz.push_back(0.f);
    sidx.push_back(0);
  }
  if (str.empty()) {
    str.push_back(make_float4(0, 0, 0, 0));
    rng.push_back(make_int2(0, 0));
  }
  if (dom.empty()) dom.push_back(make_float4(0, 0, 0, 0));
  int rc;
  if ((rc = upload(ctx, ctx->dom, dom))) return rc;
  if ((rc = upload(ctx, ctx->str, str))) return rc;
  if ((rc = upload(ctx, ctx->str_range, rng))) return rc;
  if ((rc = upload(ctx, ctx->sdom_z, sz))) return rc;
  if ((rc = upload(ctx, ctx->sdom_idx, sidx))) return rc;
  std::vector<uint8_t> clear_pad(clear);
  clear_pad.resize((clear.size() + 15) & ~(size_t)15, 0);
  if ((rc = upload(ctx, ctx->clear, clear_pad))) return rc;
  if ((rc = upload(ctx, ctx->cell_off, coff))) return rc;
  if ((rc = upload(ctx, ctx->cell_list, clist))) return rc;
  GeomDev& G = ctx->geom;
  G.dom = static_cast<const float4*>(ctx->dom.p);
  G.str = static_cast<const float4*>(ctx->str.p);
  G.str_range = static_cast<const int2*>(ctx->str_range.p);
  G.sdom_z = static_cast<const float*>(ctx->sdom_z.p);
  G.sdom_idx = static_cast<const int*>(ctx->sdom_idx.p);
  G.clear = static_cast<const uint8_t*>(ctx->clear.p);
  G.cell_off = static_cast<const uint32_t*>(ctx->cell_off.p);
  G.cell_list = static_cast<const uint16_t*>(ctx->cell_list.p);
  G.n_dom = n_dom;
  G.n_str = n_dom ? n_str : 0;
  G.nx = nx;
  G.ny = ny;
  G.r = (float)r;
  G.r2 = (float)(r * r);
  G.zpad = (float)(r + eps);
  G.gx0 = (float)(-R);
  G.gy0 = (float)(-R);
  G.inv_cell = (float)(1.0 / cell);
  G.halo = (float)halo;
  G.clear_unit = (float)unit;
  G.R = (float)R;
  G.R2 = (float)(R * R);
  G.zlo = (float)zlo;
  G.zhi = (float)zhi;
  ctx->geom_loaded = true;
  drop_graphs(ctx);
  return PP_OK;
}

int pp_load_ice(pp_ctx* ctx, const float* b_e, const float* a, int32_t n_layers,
                float depth_top_m, float dz_m, float g) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->servers > 0) return fail(ctx, PP_EINVAL, "a serving loop is attached to this context");
  if (!b_e || !a || n_layers < 1 || n_layers > kMaxLayers || !(dz_m > 0.f) ||
      !std::isfinite(dz_m) || !std::isfinite(depth_top_m) || !(g > -1.f && g < 1.f))
    return fail(ctx, PP_EINVAL, "need 1 <= n_layers <= 4096, dz > 0, -1 < g < 1");
  for (int i = 0; i < n_layers; ++i)
    if (!(b_e[i] >= 0.f) || !(a[i] >= 0.f) || !std::isfinite(b_e[i]) || !std::isfinite(a[i]))
      return fail(ctx, PP_EINVAL, "coefficients must be finite and >= 0");
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  const double gd = g;
  std::vector<float4> lay(n_layers);
  const float inf = INFINITY;
  for (int i = 0; i < n_layers; ++i) {
    const double b = ctx->cfg.scatter_coeff_is_effective ? (double)b_e[i] / (1.0 - gd) : (double)b_e[i];
    const float bf = (float)b, af = a[i];
    lay[i] = make_float4(bf, af, bf > 0.f ? (float)(1.0 / b) : inf, af > 0.f ? (float)(1.0 / (double)af) : inf);
  }
  int rc;
  if ((rc = upload(ctx, ctx->layers, lay))) return rc;
  IceDev& I = ctx->ice;
  I.layer = static_cast<const float4*>(ctx->layers.p);
  I.L = n_layers;
  I.z_top = (float)((double)ctx->cfg.depth_of_z0_m - (double)depth_top_m);
  I.dz = dz_m;
  I.g = g;
  I.c1 = (float)(1.0 - gd * gd);
  I.c2 = (float)(1.0 - gd);
  I.c3 = (float)(2.0 * gd);
  I.c4 = (float)(1.0 + gd * gd);
  I.c5 = gd != 0.0 ? (float)(1.0 / (2.0 * gd)) : 0.f;
  ctx->ice_loaded = true;
  drop_graphs(ctx);
  return PP_OK;
}

int pp_propagate(pp_ctx* ctx, uint64_t event_id, const pp_source* src, int64_t n_src,
                 uint64_t* hits, uint64_t* counts) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (n_src < 0) return fail(ctx, PP_EINVAL, "n_src < 0");
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  const int64_t begin[2] = {0, n_src};
  return batch_host(ctx, true, 1, &event_id, begin, src, hits, counts);
}

int pp_propagate_batch(pp_ctx* ctx, int32_t n_events, const uint64_t* event_ids,
                       const int64_t* src_begin, const pp_source* src, uint64_t* hits,
                       uint64_t* counts) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  return batch_host(ctx, false, n_events, event_ids, src_begin, src, hits, counts);
}

int pp_propagate_batch_async(pp_ctx* ctx, int32_t n_events, const uint64_t* d_event_ids,
                             const int64_t* d_src_begin, const pp_source* d_src, int64_t n_src,
                             uint64_t* d_hits, uint64_t* d_counts, void* stream) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  return batch_async(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits, d_counts,
                     pick_stream(ctx, stream));
}

int pp_propagate_records_async(pp_ctx* ctx, int32_t n_events, const uint64_t* d_event_ids,
                               const int64_t* d_src_begin, const pp_source* d_src, int64_t n_src,
                               uint64_t* d_hits, uint64_t* d_counts, float group_index,
                               pp_hit* d_records, uint64_t max_records, uint64_t* d_n_records,
                               void* stream) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  const RecordsOut rec{d_records, max_records, d_n_records,
                       group_index > 0.0f ? group_index : (float)kGroupIndexDefault};
  return batch_async(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits, d_counts,
                     pick_stream(ctx, stream), &rec);
}

int pp_propagate_plain_async(pp_ctx* ctx, int32_t n_events, const uint64_t* h_event_ids,
                             const int64_t* h_src_begin, const uint64_t* h_event_photons,
                             const pp_source* d_src, uint64_t* d_hits, uint64_t* d_counts,
                             void* stream) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  return plain_async(ctx, n_events, h_event_ids, h_src_begin, h_event_photons, d_src, d_hits,
                     d_counts, pick_stream(ctx, stream));
}

int pp_propagate_range_async(pp_ctx* ctx, uint64_t event_id, const pp_source* d_src,
                             int64_t n_src, uint64_t photon_begin, uint64_t photon_end,
                             int32_t accumulate, uint64_t* d_hits, uint64_t* d_counts,
                             void* stream) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  return range_async(ctx, event_id, d_src, n_src, photon_begin, photon_end, accumulate != 0,
                     d_hits, d_counts, pick_stream(ctx, stream));
}

int pp_sync(pp_ctx* ctx, void* stream) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  return sync_and_check(ctx, pick_stream(ctx, stream));
}

int pp_set_launch(pp_ctx* ctx, int32_t block_threads, int32_t blocks_per_sm,
                  int32_t refill_threshold, int32_t photons_per_lane) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (block_threads != 0 && block_threads != 128 && block_threads != 256 && block_threads != 512 &&
      block_threads != 1024)
    return fail(ctx, PP_EINVAL, "block_threads must be 128, 256, 512 or 1024");
  if (blocks_per_sm < 0 || refill_threshold < 0 || refill_threshold > 32)
    return fail(ctx, PP_EINVAL, "blocks_per_sm >= 0 and 0 <= refill_threshold <= 32");
  if (photons_per_lane < 0 || photons_per_lane > 2)
    return fail(ctx, PP_EINVAL, "photons_per_lane must be 0 (keep), 1 or 2");
  if (block_threads) ctx->block_threads = block_threads;
  ctx->blocks_per_sm = blocks_per_sm;
  if (refill_threshold) ctx->refill = refill_threshold;
  if (photons_per_lane) ctx->lane_photons = photons_per_lane;
  return PP_OK;
}

int pp_get_launch(const pp_ctx* ctx_c, int32_t* block_threads, int32_t* blocks_per_sm,
                  int32_t* refill_threshold, int32_t* photons_per_lane, int32_t* grid) {
  pp_ctx* ctx = const_cast<pp_ctx*>(ctx_c);
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (block_threads) *block_threads = ctx->block_threads;
  if (blocks_per_sm) *blocks_per_sm = ctx->blocks_per_sm;
  if (refill_threshold) *refill_threshold = ctx->refill;
  if (photons_per_lane) *photons_per_lane = ctx->lane_photons;
  if (grid) {
    *grid = 0;
    if (ctx->geom_loaded && ctx->ice_loaded) {
      DeviceScope dev_scope(ctx->cfg.device);
      PP_CUDA(dev_scope.status());
      size_t smem;
      int rc = prepare_smem(ctx, &smem, kernel_variant(ctx));
      if (!rc) rc = grid_blocks(ctx, smem, grid);
      if (rc) return rc;
    }
  }
  return PP_OK;
}

int pp_autotune_batch(pp_ctx* ctx, int32_t n_events, const uint64_t* d_event_ids,
                      const int64_t* d_src_begin, const pp_source* d_src, int64_t n_src,
                      uint64_t* d_hits, uint64_t* d_counts, void* stream, int32_t repeats,
                      int32_t* best4, float* best_ms) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  if (repeats < 1) repeats = 1;
  cudaStream_t st = pick_stream(ctx, stream);
  struct Cand {
    int bt, bps, refill, lane_photons;
  };
  // one photon per lane: refill thresholds around the measured optimum (8);
  // two photons per lane: reserved photons are cheap to hand out, so small
  // thresholds; the reserve's shared memory limits 256-thread blocks to 3-4
  // per SM, so larger blocks (tables staged once for more warps) are tried
  static const Cand cands[] = {
      {256, 0, 1, 1},  {256, 0, 2, 1},  {256, 0, 4, 1},  {256, 0, 8, 1},  {256, 0, 16, 1},
      {256, 0, 32, 1}, {256, 5, 4, 1},  {256, 5, 8, 1},  {256, 5, 16, 1}, {256, 6, 4, 1},
      {256, 6, 8, 1},  {256, 6, 16, 1}, {128, 0, 4, 1},  {128, 0, 8, 1},  {128, 0, 16, 1},
      {512, 0, 8, 1},  {512, 0, 16, 1}, {1024, 0, 16, 1},
      {256, 0, 1, 2},  {256, 0, 2, 2},  {256, 0, 4, 2},  {256, 3, 1, 2},  {256, 3, 2, 2},
      {256, 3, 4, 2},  {512, 0, 1, 2},  {512, 0, 2, 2},  {512, 0, 4, 2},  {1024, 0, 1, 2},
      {1024, 0, 2, 2}, {1024, 0, 4, 2}};
  const Cand keep{ctx->block_threads, ctx->blocks_per_sm, ctx->refill, ctx->lane_photons};
  const bool keep_timing = ctx->timing, keep_graphs = ctx->graphs;
  ctx->timing = false;
  ctx->graphs = false;
  cudaEvent_t e0, e1;
  PP_CUDA(cudaEventCreate(&e0));
  PP_CUDA(cudaEventCreate(&e1));
  float best = 3.4e38f;
  Cand win = keep;
  int rc = PP_OK;
  for (const Cand& c : cands) {
    ctx->block_threads = c.bt;
    ctx->blocks_per_sm = c.bps;
    ctx->refill = c.refill;
    ctx->lane_photons = c.lane_photons;
    // warm-up launch, then the timed ones
    rc = batch_async(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits, d_counts, st);
    if (rc) break;
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = PP_ECUDA; break; }
    for (int r = 0; r < repeats && !rc; ++r)
      rc = batch_async(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits, d_counts, st);
    if (rc) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(ctx, PP_ECUDA, "autotune timing failed");
      break;
    }
    ms /= repeats;
    if (ms < best) {
      best = ms;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->timing = keep_timing;
  ctx->graphs = keep_graphs;
  const Cand& use = rc ? keep : win;
  ctx->block_threads = use.bt;
  ctx->blocks_per_sm = use.bps;
  ctx->refill = use.refill;
  ctx->lane_photons = use.lane_photons;
  if (rc) return rc;
  if (best4) {
    best4[0] = win.bt;
    best4[1] = win.bps;
    best4[2] = win.refill;
    best4[3] = win.lane_photons;
  }
  if (best_ms) *best_ms = best;
  return PP_OK;
}

int pp_set_graphs(pp_ctx* ctx, int32_t enable) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  ctx->graphs = enable != 0;
  if (!ctx->graphs) drop_graphs(ctx);
  return PP_OK;
}

int pp_set_hit_acceptance(pp_ctx* ctx, const float* coeffs, int32_t n) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (n < 0 || n > PP_MAX_ACCEPT_COEFFS || (n > 0 && !coeffs))
    return fail(ctx, PP_EINVAL, "acceptance: 0 <= n <= 8 coefficients");
  for (int32_t i = 0; i < n; ++i)
    if (!std::isfinite(coeffs[i])) return fail(ctx, PP_EINVAL, "acceptance: non-finite coefficient");
  ctx->n_accept = n;
  for (int i = 0; i < PP_MAX_ACCEPT_COEFFS; ++i) ctx->accept[i] = i < n ? coeffs[i] : 0.0f;
  ctx->epoch += 1;  // captured graphs hold the old run parameters
  return PP_OK;
}

int pp_get_memory(pp_ctx* ctx, uint64_t* device_bytes, uint64_t* n_allocations) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (device_bytes) *device_bytes = ctx->device_bytes;
  if (n_allocations) *n_allocations = ctx->n_allocations;
  return PP_OK;
}

int pp_set_kernel_timing(pp_ctx* ctx, int32_t enable) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->timing = enable != 0;
  return PP_OK;
}

int pp_get_kernel_time(pp_ctx* ctx, double* total_ms, uint64_t* n_timed, uint64_t* n_kernels) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  double sum = 0.0;
  const uint64_t n = ctx->pending.size();
  for (auto& pr : ctx->pending) {
    PP_CUDA(cudaEventSynchronize(pr.second));
    float ms = 0.f;
    PP_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
    sum += ms;
    ctx->event_pool.push_back(pr.first);
    ctx->event_pool.push_back(pr.second);
  }
  ctx->pending.clear();
  if (total_ms) *total_ms = sum;
  if (n_timed) *n_timed = n;
  if (n_kernels) *n_kernels = ctx->kernels_launched;
  ctx->kernels_launched = 0;
  return PP_OK;
}

int pp_get_path_stats(pp_ctx* ctx, uint64_t* out4) {
  if (!ctx || !out4) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  PP_CUDA(cudaStreamSynchronize(ctx->stream));
  PP_CUDA(cudaDeviceSynchronize());
  PP_CUDA(cudaMemcpy(out4, ctx->stats.p, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  PP_CUDA(cudaMemset(ctx->stats.p, 0, 4 * sizeof(uint64_t)));
  return PP_OK;
}

int pp_get_world(const pp_ctx* ctx, float* out3) {
  if (!ctx || !out3) return PP_EINVAL;
  if (!ctx->geom_loaded) return PP_ENOTLOADED;
  out3[0] = ctx->geom.R;
  out3[1] = ctx->geom.zlo;
  out3[2] = ctx->geom.zhi;
  return PP_OK;
}

int pp_debug_philox(pp_ctx* ctx, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                    int64_t n) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(ctx, PP_EINVAL, "bad arguments");
  if (n == 0) return PP_OK;
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  int rc;
  if ((rc = ensure(ctx, ctx->s_misc1, 16 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc2, 8 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc3, 16 * (size_t)n))) return rc;
  cudaStream_t st = ctx->stream;
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc1.p, ctr, 16 * n, cudaMemcpyHostToDevice, st));
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc2.p, key, 8 * n, cudaMemcpyHostToDevice, st));
  PP_CUDA(launch_philox(static_cast<uint32_t*>(ctx->s_misc1.p), static_cast<uint32_t*>(ctx->s_misc2.p),
                        static_cast<uint32_t*>(ctx->s_misc3.p), n, st));
  PP_CUDA(cudaMemcpyAsync(out, ctx->s_misc3.p, 16 * n, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaStreamSynchronize(st));
  return PP_OK;
}

int pp_debug_trace(pp_ctx* ctx, uint64_t event_id, const pp_source* src, int64_t n_src,
                   const uint64_t* photon_ids, int64_t n, int32_t n_trace, int32_t* outcome,
                   int64_t* n_steps, float* birth, float* trace) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  if (n_src < 1 || n < 0 || n_trace < 0 || !src || (n > 0 && (!photon_ids || !outcome || !n_steps)) ||
      (n_trace > 0 && !trace) || n_src > kMaxSources)
    return fail(ctx, PP_EINVAL, "bad arguments");
  if ((rc = check_sources(ctx, src, n_src))) return rc;
  if (n == 0) return PP_OK;
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  cudaStream_t st = ctx->stream;
  if ((rc = ensure(ctx, ctx->s_src, sizeof(pp_source) * n_src))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc1, 8 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc2, 4 * (size_t)n + 8 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc3, 24 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc4, 12 * (size_t)n * std::max(n_trace, 1)))) return rc;
  if ((rc = ensure_scratch(ctx, n_src, false))) return rc;
  size_t smem;
  if ((rc = prepare_smem(ctx, &smem, 0))) return rc;
  PP_CUDA(cudaMemcpyAsync(ctx->s_src.p, src, sizeof(pp_source) * n_src, cudaMemcpyHostToDevice, st));
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc1.p, photon_ids, 8 * n, cudaMemcpyHostToDevice, st));
  const pp_source* d_src = static_cast<const pp_source*>(ctx->s_src.p);
  PP_CUDA(launch_expand(d_src, n_src, nullptr, nullptr, 1, expand_bufs(ctx, false), st));
  const WorkDev w = work_desc(ctx, d_src, n_src, false, nullptr, nullptr, nullptr, nullptr,
                              (uint32_t)event_id);
  int* d_out = static_cast<int*>(ctx->s_misc2.p);
  int64_t* d_ns = reinterpret_cast<int64_t*>(static_cast<char*>(ctx->s_misc2.p) + ((4 * n + 7) & ~7));
  float* d_birth = static_cast<float*>(ctx->s_misc3.p);
  float* d_tr = n_trace > 0 ? static_cast<float*>(ctx->s_misc4.p) : nullptr;
  PP_CUDA(launch_trace(ctx->ice, ctx->geom, w, run_params(ctx), static_cast<uint64_t*>(ctx->s_misc1.p),
                       n, n_trace, d_out, d_ns, d_birth, d_tr, smem, st));
  PP_CUDA(cudaMemcpyAsync(outcome, d_out, 4 * n, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaMemcpyAsync(n_steps, d_ns, 8 * n, cudaMemcpyDeviceToHost, st));
  if (birth) PP_CUDA(cudaMemcpyAsync(birth, d_birth, 24 * n, cudaMemcpyDeviceToHost, st));
  if (n_trace > 0)
    PP_CUDA(cudaMemcpyAsync(trace, d_tr, 12 * (size_t)n * n_trace, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaStreamSynchronize(st));
  return PP_OK;
}

int pp_debug_scatter(pp_ctx* ctx, const float* dir, const uint32_t* words, float* out, int64_t n) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->ice_loaded) return fail(ctx, PP_ENOTLOADED, "load ice first");
  if (n < 0 || (n > 0 && (!dir || !words || !out))) return fail(ctx, PP_EINVAL, "bad arguments");
  if (n == 0) return PP_OK;
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  cudaStream_t st = ctx->stream;
  int rc;
  if ((rc = ensure(ctx, ctx->s_misc1, 12 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc2, 8 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc3, 12 * (size_t)n))) return rc;
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc1.p, dir, 12 * n, cudaMemcpyHostToDevice, st));
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc2.p, words, 8 * n, cudaMemcpyHostToDevice, st));
  PP_CUDA(launch_scatter(ctx->ice, static_cast<float*>(ctx->s_misc1.p),
                         static_cast<uint32_t*>(ctx->s_misc2.p), static_cast<float*>(ctx->s_misc3.p),
                         n, st));
  PP_CUDA(cudaMemcpyAsync(out, ctx->s_misc3.p, 12 * n, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaStreamSynchronize(st));
  return PP_OK;
}

int pp_debug_gemm(pp_ctx* ctx, const uint16_t* A, const uint16_t* B, int32_t M, int32_t N,
                  int32_t K, float* C) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!A || !B || !C || M < 1 || N < 16 || N > 256 || N % 16 || K < 16 || K % 16)
    return fail(ctx, PP_EINVAL, "need M >= 1, 16 <= N <= 256 (multiple of 16), K multiple of 16");
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  cudaStream_t st = ctx->stream;
  int rc;
  const size_t a = 2 * (size_t)M * K, b = 2 * (size_t)N * K, c = 4 * (size_t)M * N;
  if ((rc = ensure(ctx, ctx->s_misc1, a)) || (rc = ensure(ctx, ctx->s_misc2, b)) ||
      (rc = ensure(ctx, ctx->s_misc3, c)))
    return rc;
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc1.p, A, a, cudaMemcpyHostToDevice, st));
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc2.p, B, b, cudaMemcpyHostToDevice, st));
  mlp::GemmArgs g{};
  g.A = static_cast<const __nv_bfloat16*>(ctx->s_misc1.p);
  g.B = static_cast<const __nv_bfloat16*>(ctx->s_misc2.p);
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = K;
  g.ldb = K;
  g.ldc = N;
  g.bn = N;
  g.Cf = static_cast<float*>(ctx->s_misc3.p);
  g.err = static_cast<int*>(ctx->err.p);
  PP_CUDA(mlp::launch_gemm(g, st));
  PP_CUDA(cudaMemcpyAsync(C, ctx->s_misc3.p, c, cudaMemcpyDeviceToHost, st));
  return sync_and_check(ctx, st);
}

int pp_debug_first_hit(pp_ctx* ctx, const float* seg, int64_t n, int32_t mode, int32_t* dom,
                       float* t) {
  if (!ctx) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  int rc;
  if ((rc = check_loaded(ctx))) return rc;
  if (n < 0 || (n > 0 && (!seg || !dom || !t)) || (mode != 0 && mode != 1))
    return fail(ctx, PP_EINVAL, "bad arguments");
  if (n == 0) return PP_OK;
  DeviceScope dev_scope(ctx->cfg.device);
  PP_CUDA(dev_scope.status());
  cudaStream_t st = ctx->stream;
  if ((rc = ensure(ctx, ctx->s_misc1, 28 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc2, 4 * (size_t)n))) return rc;
  if ((rc = ensure(ctx, ctx->s_misc3, 4 * (size_t)n))) return rc;
  size_t smem;
  if ((rc = prepare_smem(ctx, &smem, 0))) return rc;
  PP_CUDA(cudaMemcpyAsync(ctx->s_misc1.p, seg, 28 * n, cudaMemcpyHostToDevice, st));
  PP_CUDA(launch_first_hit(ctx->geom, ctx->ice, static_cast<float*>(ctx->s_misc1.p), n, mode,
                           static_cast<int*>(ctx->s_misc2.p), static_cast<float*>(ctx->s_misc3.p),
                           smem, st));
  PP_CUDA(cudaMemcpyAsync(dom, ctx->s_misc2.p, 4 * n, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaMemcpyAsync(t, ctx->s_misc3.p, 4 * n, cudaMemcpyDeviceToHost, st));
  PP_CUDA(cudaStreamSynchronize(st));
  return PP_OK;
}

}  // extern "C"
