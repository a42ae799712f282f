// Internal interface between the C ABI (pp_capi.cu) and the kernels
// (pp_kernels.cu).  Not installed, not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "pp.h"

namespace ppk {

// Makes `device` current for the enclosing scope and gives the calling
// thread back its own current device on exit: an entry point never leaves a
// host thread that drives another GPU switched to this library's device.
class DeviceScope {
 public:
  explicit DeviceScope(int device) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      (void)cudaGetLastError();
      prev_ = -1;
    }
    status_ = (prev_ == device) ? cudaSuccess : cudaSetDevice(device);
    restore_ = status_ == cudaSuccess && prev_ >= 0 && prev_ != device;
  }
  ~DeviceScope() {
    if (restore_) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  cudaError_t status() const { return status_; }

 private:
  int prev_ = -1;
  bool restore_ = false;
  cudaError_t status_ = cudaSuccess;
};

constexpr int kMaxLayers = 4096;
constexpr int kMaxStrings = 4096;
constexpr int kMaxCells = 32768;         // u8 clearance grid staged in shared memory
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;            // sources per scan thread
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kTopThreads = 1024;
constexpr int kTopItems = 16;
constexpr int64_t kMaxSources = (int64_t)kScanTile * kTopThreads * kTopItems;  // 33.5 M
constexpr int kSmallThreads = 1024;      // fused single-block expansion
constexpr int kSmallItems = 8;
constexpr int64_t kSmallMax = (int64_t)kSmallThreads * kSmallItems;

// Per-step outcome of a photon (>= 0: the DOM it hit).
constexpr int kScattered = -100;  // the step ended in a scatter; the photon goes on
constexpr int kAbsorbed = PP_OUT_ABSORBED;
constexpr int kEscaped = PP_OUT_ESCAPED;
constexpr int kTruncated = PP_OUT_TRUNCATED;

// Error flag bits (latched in device memory, read by pp_sync).
constexpr int kErrBadSource = 1;
constexpr int kErrBadIndex = 2;

// Ice table as the kernels read it: per layer (b, a, 1/b, 1/a) with b the
// geometric scattering coefficient; 1/x is +inf where x is 0.
struct IceDev {
  const float4* layer;
  int L;
  float z_top;   // z of the top of layer 0
  float dz;
  float g;
  float c1, c2, c3, c4, c5;   // HG: 1-g^2, 1-g, 2g, 1+g^2, 1/(2g)
};

// Detector tables.  DOMs are grouped by string; each string is bounded by a
// vertical cylinder (cx, cy, radius incl. DOM radius and a margin); the DOMs
// of a string are listed by ascending z.  A 2-D cell grid holds for each cell
// a lower bound of the horizontal distance from any point of the cell to any
// string cylinder ("clearance", in units of clear_unit) and the strings
// within `halo` of the cell.
struct GeomDev {
  const float4* dom;        // [n_dom] (x, y, z, 0)
  const float4* str;        // [n_str] (cx, cy, radius, 0)
  const int2* str_range;    // [n_str] (first, count) into sdom_*
  const float* sdom_z;      // [n_dom] z, per string ascending
  const int* sdom_idx;      // [n_dom] DOM index, same order
  const uint8_t* clear;     // [ny][nx]
  const uint32_t* cell_off; // [nx*ny + 1] into cell_list
  const uint16_t* cell_list;
  int n_dom, n_str, nx, ny;
  float r, r2, zpad;        // DOM radius, r^2, z window padding
  float gx0, gy0, inv_cell, halo, clear_unit;
  float R, R2, zlo, zhi;    // world cylinder
};

// Per-source event record written by the expansion (batch mode): the
// event-local photon id of the source's first photon, the event id's low word
// (Philox key) and the event slot (row of the outputs).
struct SrcAux {
  unsigned long long base;
  uint32_t ev_lo;
  uint32_t ev;
};

// One propagation launch's work description.
struct WorkDev {
  const pp_source* src;       // batch sources
  const uint64_t* off;        // [n_src + 1] photon prefix over the batch
  const uint32_t* chunk_src;  // [n_src + 2] first source of each photon chunk
  const SrcAux* aux;          // [n_src] event record of each source (NULL: single event)
  const uint64_t* meta;       // [0] total photons, [1] chunk log2
  unsigned long long* work;   // persistent work counter (zeroed before launch)
  unsigned long long* hits;   // [n_events][n_dom]
  unsigned long long* counts; // [n_events][4]
  int* err;
  unsigned long long* stats;  // [4] steps, layer crossings, births, 0 (persistent kernel)
  int n_src;
  uint32_t single_event_lo;   // event id (low word) in single-event mode
  uint64_t g_begin, g_end;    // persistent kernel: batch photon range to run
  // compact hit records (records kernel variant only): one pp_hit per hit,
  // appended at an atomic cursor; records past max_records are counted, not written
  pp_hit* records;
  unsigned long long* n_records;
  uint64_t max_records;
};

struct RunDev {
  // Philox key schedule of the run: round r's key words (seed lo + r W0,
  // seed hi + r W1), precomputed on the host.  The key is the same for every
  // photon (the event id sits in the counter), so the rounds read their keys
  // as kernel-parameter constants instead of bumping a per-lane key.
  uint32_t key_x[10], key_y[10];
  uint32_t max_steps;
  float cos_cherenkov, sin_cherenkov;
  int refill;                 // persistent: refill once this many lanes are idle (with the
                              // reserve: take reserved photons once this many are idle)
  float ns_per_m_emit;        // hit time: emission offset along the segment at c (ns / m)
  float ns_per_m_path;        // hit time: photon path at the group velocity (ns / m)
  int n_accept;               // hit records: acceptance polynomial in the direction's z
  float accept[PP_MAX_ACCEPT_COEFFS];
};

// Shared-memory footprint of the tables the propagation kernels stage
// (layers float4, strings float4 + int2, u8 clearance cells; 16-byte multiple).
__host__ __device__ inline size_t tables_bytes(int n_layers, int n_str, int n_cells) {
  const size_t b = (size_t)n_layers * 16 + (size_t)n_str * 24 + (size_t)n_cells;
  return (b + 15) & ~(size_t)15;
}
size_t tables_smem_bytes(const IceDev& ice, const GeomDev& geom);

// Photon reserve of the persistent kernel (two photons per lane): each warp
// keeps up to kReserveCap born photons in shared memory, kReserveWords 32-bit
// words each (position, direction, tau_a, layer, id words, event slot; the
// records variant adds the emission offset and the source index), laid out
// word-major so that consecutive slots fall in consecutive banks.
constexpr int kReserveCap = 48;
constexpr int kReserveWords = 12;
constexpr int kReserveWordsRecords = 14;
inline size_t reserve_smem_bytes(int block_threads, bool records) {
  return (size_t)(block_threads / 32) * kReserveCap *
         (records ? kReserveWordsRecords : kReserveWords) * 4;
}

// Scratch needed by the expansion for n_src sources.
struct ExpandBufs {
  uint64_t* off;          // n_src + 1
  uint32_t* chunk_src;    // n_src + 2
  SrcAux* aux;            // n_src (NULL in single-event mode)
  uint64_t* bsum;         // ceil(n_src / kScanTile)
  uint64_t* meta;         // 2
};

// a1: exclusive prefix of n_photons over the sources, photon-chunk table and
// source -> event map.  src_begin/n_events may be NULL/0 (single event).
cudaError_t launch_expand(const pp_source* src, int64_t n_src, const int64_t* src_begin,
                          const uint64_t* event_ids, int n_events, const ExpandBufs& b,
                          cudaStream_t st);

// a2..a8 for the photons of the work description.
//   persistent = false: one thread per photon, `n_photons_host` photons
//   persistent = true : grid_blocks persistent blocks with warp refill
// variant selects the register budget of the persistent kernel: 0 = any block
// size (up to 64 registers), 5 / 6 = 256-thread blocks, 5 / 6 resident per SM;
// kVariantRecords = variant 0 that also writes compact hit records;
// + kVariantReserve: the same kernel with a per-warp photon reserve (two
// photons per lane: births of whole warps into shared memory, idle lanes
// take the next reserved photon).
constexpr int kVariantRecords = 7;
constexpr int kPlainThreads = 256;  // block size of the plain (one thread per photon) path
constexpr int kVariantReserve = 16;

// Hit times: light speed in vacuum, and the group index used unless the
// caller gives one (the paper gives none; 1.35 is a typical value for ice in
// the blue, a reading).
constexpr double kLightSpeedMperNs = 0.299792458;
constexpr double kGroupIndexDefault = 1.35;
cudaError_t launch_propagate(bool persistent, const IceDev& ice, const GeomDev& geom,
                             const WorkDev& work, const RunDev& run, int block_threads,
                             int grid_blocks, uint64_t n_photons_host, size_t smem,
                             cudaStream_t st, int variant = 0);

cudaError_t set_propagate_smem_limit(size_t smem);
cudaError_t propagate_occupancy(int block_threads, size_t smem, int variant, int* blocks_per_sm);

cudaError_t launch_trace(const IceDev& ice, const GeomDev& geom, const WorkDev& work,
                         const RunDev& run, const uint64_t* ids, int64_t n, int n_trace,
                         int* outcome, int64_t* n_steps, float* birth, float* trace,
                         size_t smem, cudaStream_t st);

// *first_bad = min(*first_bad, base + index of each malformed source)
cudaError_t launch_check_sources(const pp_source* src, int64_t n, int64_t base,
                                 unsigned long long* first_bad, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                          cudaStream_t st);

cudaError_t launch_scatter(const IceDev& ice, const float* dir, const uint32_t* words, float* out,
                           int64_t n, cudaStream_t st);

cudaError_t launch_first_hit(const GeomDev& geom, const IceDev& ice, const float* seg, int64_t n,
                             int mode, int* dom, float* t, size_t smem, cudaStream_t st);

// What a launch needs from a context, for entry points defined outside
// pp_capi.cu.  with_launch_view locks the context, checks that geometry and
// ice are loaded, prepares the kernels' shared-memory limit and the persistent
// grid, and calls fn with the view (fn's return value is returned).
struct LaunchView {
  pp_ctx* ctx;
  int device;
  cudaStream_t stream;
  IceDev ice;
  GeomDev geom;
  RunDev run;
  int block_threads;
  int grid_blocks;
  int variant;
  int scatter_effective;  // the context's scatter_coeff_is_effective
  size_t smem;
  int* err;
  unsigned long long* stats;
  int fail(int code, const char* msg) const;
  int cuda_fail(cudaError_t e, const char* where) const;
};

int with_launch_view(pp_ctx* ctx, const std::function<int(const LaunchView&)>& fn);

// ---- serving: the device-resident request ring ------------------------------
// One admitted request (a bunch of sources of one event) in the ring the
// serving kernel pulls photons from; request q lives in slot q % cap.  The
// host fills a slot in two copies before it publishes the request: first
// everything but `claimed` (done = 0), then `claimed` = (q mod 2^28) << 36,
// which arms the slot.  Warps claim photons by adding 32 to `claimed`: the
// high bits say which request the claim went to, the low bits where it
// starts.  A claim is kept only if the slot's seq matches its high bits and
// it starts below the total, so a warp still looking at a slot's previous
// request can never take photons twice.
struct ServeReq {
  unsigned long long claimed;  // (request number mod 2^28) << 36 | photons claimed
  unsigned long long done;     // photons tallied so far
  uint64_t total;              // photons of the request (0 < total < 2^35)
  uint64_t src_off;            // its first source in the source arena
  uint64_t off_off;            // its photon prefix (n_src + 1 entries) in the prefix arena
  uint64_t chunk_off;          // its photon-chunk table in the chunk arena
  uint32_t n_src, chunk_log2;  // as the batch expansion's meta
  uint32_t event_lo;           // event id, low word (the Philox key word)
  uint32_t seq;                // request number (low word)
};
static_assert(sizeof(ServeReq) == 64, "request entry layout");

constexpr int kServeOffsetBits = 36;
constexpr int kServeSeqBits = 28;
constexpr uint64_t kServeMaxPhotons = 1ull << 35;  // headroom above a total for late claims
constexpr int kServeMaxRequests = 1 << 16;         // ring capacity limit (a power of two)

struct ServeDev {
  ServeReq* req;                     // [cap] (cap a power of two)
  int cap;
  const unsigned long long* tail;    // requests published (written by host copies)
  unsigned long long* head;          // oldest request that may have unclaimed photons
  const pp_source* src;              // source arena
  const uint64_t* off;               // prefix arena
  const uint32_t* chunk;             // chunk arena
  unsigned long long* hits;          // [cap][n_dom]
  unsigned long long* counts;        // [cap][4] absorbed, escaped, truncated, steps
  volatile uint32_t* done_flag;      // host-mapped [cap]: seq + 1 once tallied
  int* err;
  const int* may_leave;              // 1 while the host holds no unfinished request
                                     // (written by host copies)
  int* closing;                      // set by the warp that ends the launch; cleared by
                                     // the host before each launch
  uint64_t idle_ns;                  // an idle warp closes the launch after this long, once
                                     // may_leave is set
  uint64_t max_ns;                   // the launch closes this long after its start
};

// The serving kernel: persistent blocks (1024 threads, photon reserve) that
// take photons from published requests until idle.
cudaError_t launch_serve(const IceDev& ice, const GeomDev& geom, const ServeDev& sv,
                         const RunDev& run, int grid_blocks, size_t smem, cudaStream_t st);
cudaError_t serve_occupancy(size_t smem, int* blocks_per_sm);
constexpr int kServeThreads = 1024;

// Servers that hold a LaunchView of the context (its table pointers): while
// any is attached the context refuses to load new geometry or ice.
void attach_server(pp_ctx* ctx, int delta);

// Adds n to the context's count of launched kernels (pp_stats); the caller
// holds the context's lock (inside with_launch_view).
void count_launches(pp_ctx* ctx, int n);

// pp_noalloc.cu: looks up the device address of the no-allocation entry
// point's static scratch array on `device` (which must be current) and keeps
// it for that device, replacing an earlier one.  Called by pp_create, so a
// context created after a device reset never sees a stale address.
cudaError_t noalloc_setup(int device);

}  // namespace ppk
