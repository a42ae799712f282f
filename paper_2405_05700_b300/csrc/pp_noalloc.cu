// pp_propagate_noalloc: one event through the expansion and the persistent
// propagation kernel without allocating any device memory during the call.
//
// The scratch these kernels need (photon prefix sums, the photon-chunk table,
// the expansion totals and the work counter) lives in one file-scope device
// array below instead of context buffers grown with cudaMalloc.  Every GPU
// that loads this library holds the array until the process exits.  In host
// code the array's name is only a stand-in for the symbol, not a device
// address: the address the kernels get comes from cudaGetSymbolAddress, taken
// with the device current when a context is created on it (pp_create calls
// noalloc_setup), and again by the first call on a device that has none.
#include <cuda_runtime.h>

#include <mutex>

#include "pp.h"
#include "pp_internal.h"

namespace {

constexpr int64_t kMaxSrc = PP_NOALLOC_MAX_SOURCES;
static_assert(kMaxSrc <= ppk::kSmallMax, "single-block expansion only");

// Byte layout of the scratch array (each part on its own 256-byte boundary).
constexpr size_t kOffBytes = ((sizeof(uint64_t) * (kMaxSrc + 1) + 255) / 256) * 256;
constexpr size_t kChunkBytes = ((sizeof(uint32_t) * (kMaxSrc + 2) + 255) / 256) * 256;
constexpr size_t kOffAt = 0;
constexpr size_t kChunkAt = kOffAt + kOffBytes;
constexpr size_t kMetaAt = kChunkAt + kChunkBytes;   // 2 x u64
constexpr size_t kWorkAt = kMetaAt + 256;            // 1 x u64, zeroed per call
constexpr size_t kBsumAt = kWorkAt + 256;            // unused by the single-block path
constexpr size_t kScratchBytes = kBsumAt + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

cudaError_t lookup(int device) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[device] = p;
  return cudaSuccess;
}

// Device address of the scratch array on `device` (current): the one the
// last set-up found there, else looked up now.
cudaError_t scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[device]) {
    const cudaError_t e = lookup(device);
    if (e != cudaSuccess) return e;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return cudaSuccess;
}

}  // namespace

namespace ppk {

cudaError_t noalloc_setup(int device) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  return lookup(device);
}

}  // namespace ppk

extern "C" int pp_propagate_noalloc(pp_ctx* ctx, uint64_t event_id, const pp_source* d_src,
                                    int64_t n_src, uint64_t* d_hits, uint64_t* d_counts,
                                    void* stream) {
  if (!ctx) return PP_EINVAL;
  return ppk::with_launch_view(ctx, [&](const ppk::LaunchView& v) -> int {
    if (n_src < 0 || n_src > kMaxSrc)
      return v.fail(PP_EINVAL, "pp_propagate_noalloc takes 0..8192 sources per call "
                               "(PP_NOALLOC_MAX_SOURCES); split the event or use "
                               "pp_propagate_batch_async");
    if (!d_hits || !d_counts || (n_src > 0 && !d_src))
      return v.fail(PP_EINVAL, "null device pointer");
    unsigned char* base = nullptr;  // with_launch_view made v.device current
    cudaError_t e = scratch_address(v.device, &base);
    if (e != cudaSuccess) return v.cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : v.stream;
    if (v.geom.n_dom)
      e = cudaMemsetAsync(d_hits, 0, sizeof(uint64_t) * (size_t)v.geom.n_dom, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * 4, st);
    if (e != cudaSuccess) return v.cuda_fail(e, "cudaMemsetAsync(outputs)");
    if (n_src == 0) return PP_OK;
    ppk::ExpandBufs b;
    b.off = reinterpret_cast<uint64_t*>(base + kOffAt);
    b.chunk_src = reinterpret_cast<uint32_t*>(base + kChunkAt);
    b.aux = nullptr;
    b.bsum = reinterpret_cast<uint64_t*>(base + kBsumAt);
    b.meta = reinterpret_cast<uint64_t*>(base + kMetaAt);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(base + kWorkAt);
    e = cudaMemsetAsync(work, 0, sizeof(uint64_t), st);  // the counter starts at 0 each call
    if (e == cudaSuccess) e = ppk::launch_expand(d_src, n_src, nullptr, nullptr, 1, b, st);
    if (e != cudaSuccess) return v.cuda_fail(e, "noalloc expansion");
    ppk::count_launches(v.ctx, 1);
    ppk::WorkDev w{};
    w.src = d_src;
    w.off = b.off;
    w.chunk_src = b.chunk_src;
    w.aux = nullptr;
    w.meta = b.meta;
    w.work = work;
    w.hits = reinterpret_cast<unsigned long long*>(d_hits);
    w.counts = reinterpret_cast<unsigned long long*>(d_counts);
    w.err = v.err;
    w.stats = v.stats;
    w.n_src = (int)n_src;
    w.single_event_lo = (uint32_t)event_id;
    w.g_begin = 0;
    w.g_end = ~0ull;
    e = ppk::launch_propagate(true, v.ice, v.geom, w, v.run, v.block_threads, v.grid_blocks, 0,
                              v.smem, st, v.variant);
    if (e != cudaSuccess) return v.cuda_fail(e, "noalloc propagation");
    ppk::count_launches(v.ctx, 1);
    return PP_OK;
  });
}
