/*
 * pp.h -- C ABI of the B300 photon propagator.
 *
 * Monte Carlo propagation of photons from light sources ("photon emitting
 * steps", paper Sec. 4) through ice described in 10 m depth layers with
 * per-layer scattering and absorption coefficients, until each photon reaches
 * a detector module (DOM), is absorbed, or leaves the simulated volume
 * (paper Sec. 2: distance to the next scatter drawn by Monte Carlo, a new
 * angle from the scattering physics, repeated until the photon meets a DOM or
 * is absorbed; photons are independent, "embarrassingly parallel").
 *
 * Conventions for every entry point:
 *   - Return 0 (PP_OK) or a negative PP_E* code; pp_last_error() gives a
 *     message for the context.  No C++ exception crosses this ABI.
 *   - Host pointers are caller-owned, read (or written) only during the call.
 *   - Device pointers ("d_" prefix) are caller-owned device memory on the
 *     context's device; *_async entry points enqueue work on the given CUDA
 *     stream (NULL: the context's stream) and return without synchronising;
 *     the caller keeps the buffers alive until that work completes.
 *   - Memory the library needs beyond inputs and outputs (geometry tables,
 *     prefix sums, work counters, staging copies of host inputs) is owned by
 *     the context, allocated with cudaMalloc, grown on demand and freed by
 *     pp_destroy().
 *   - Results depend only on (seed, event id, the event's sources, geometry,
 *     ice, settings): never on batching, launch shape or timing.  Random
 *     numbers are Philox4x32-10 keyed by the 64-bit seed with counter
 *     (photon id, step, event id), and tallies are integer atomics, so hits
 *     + absorbed + escaped equals the number of emitted photons exactly.
 *   - Calls on one context are serialised by the library (a mutex).
 *
 * Coordinates: metres, right-handed, z up; depth = depth_of_z0_m - z.
 */
#ifndef PP_H_
#define PP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PP_OK 0
#define PP_EINVAL (-1)      /* bad argument (null pointer, size, non-finite value) */
#define PP_ENOTLOADED (-2)  /* geometry or ice not loaded yet */
#define PP_EBUDGET (-3)     /* request larger than the configured budget */
#define PP_ETIMEDOUT (-4)   /* a bounded wait ran out */
#define PP_ECUDA (-5)       /* a CUDA runtime call failed (message in pp_last_error) */
#define PP_EDEVICE (-6)     /* a kernel raised its error flag (bad input seen on device) */
#define PP_ENOMEM (-7)      /* device allocation failed */
#define PP_ENODEV (-8)      /* no usable CUDA device */

/* Source types.  ISO_POINT and CASCADE emit isotropically from a point on the
 * segment; CHERENKOV emits on a 41 degree cone about the segment direction. */
#define PP_SRC_ISO_POINT 0u
#define PP_SRC_CHERENKOV 1u
#define PP_SRC_CASCADE 2u

/* Photon outcome codes of pp_debug_trace (a value >= 0 is the DOM index). */
#define PP_OUT_ABSORBED (-1)
#define PP_OUT_ESCAPED (-2)
#define PP_OUT_TRUNCATED (-3)

typedef struct pp_ctx pp_ctx; /* opaque, library-owned */

typedef struct pp_config {
  int32_t device;                     /* CUDA device ordinal */
  uint32_t max_steps;                 /* step cap per photon; reaching it counts as absorbed
                                         and as truncated (default 100000) */
  uint64_t seed;                      /* Philox key (low word, high word) */
  float world_margin_m;               /* world cylinder = DOM extent + margin (default 100) */
  float depth_of_z0_m;                /* depth of the z = 0 plane (default 1950) */
  int32_t scatter_coeff_is_effective; /* 1 (default): b_e is the effective coefficient and the
                                         geometric one is b_e / (1 - g); 0: b_e is used as is */
  int32_t reserved;
  void* stream;                       /* cudaStream_t for the context's work; NULL: a stream
                                         the context creates */
} pp_config;

/* One light source, 40 bytes: photons are born uniformly along the segment
 * [x, x + length * d] (a point when length is 0). */
typedef struct pp_source {
  float x, y, z;    /* start point (m) */
  float dx, dy, dz; /* direction of the emitting segment (normalised on use) */
  float length;     /* segment length (m), >= 0 */
  uint32_t type;    /* PP_SRC_* */
  uint64_t n_photons;
} pp_source;

/* Fills *cfg with the defaults listed above.  Returns PP_EINVAL on NULL. */
int pp_config_default(pp_config* cfg);

/* Creates a context on cfg->device.  *out receives the context.
 * Errors: PP_EINVAL, PP_ENODEV, PP_ECUDA. */
int pp_create(const pp_config* cfg, pp_ctx** out);

/* Frees the context and all device memory it owns.  NULL is accepted. */
int pp_destroy(pp_ctx* ctx);

/* Message for the last error raised on this context (never NULL). */
const char* pp_last_error(const pp_ctx* ctx);

/* Text for a PP_E* code (never NULL). */
const char* pp_strerror(int code);

/* Loads the detector (paper Sec. 1: DOMs on vertical strings between 1450 m
 * and 2450 m depth).
 *   xyz        [n_dom][3] float32 DOM centres (m), host memory
 *   string_id  [n_dom] int32 string of each DOM (DOMs of one string should sit
 *              near one vertical line; any grouping gives the same results,
 *              this one is fast)
 *   n_dom      0 <= n_dom <= 65535
 *   dom_radius sphere radius (m), > 0
 * Builds the per-string tables, the 2-D cell grid used by the hit test, and
 * the world cylinder (radius = max DOM distance from the z axis + margin,
 * z range = DOM z range +- margin).  Errors: PP_EINVAL, PP_ENOMEM, PP_ECUDA. */
int pp_load_geometry(pp_ctx* ctx, const float* xyz, const int32_t* string_id, int32_t n_dom,
                     float dom_radius);

/* Loads the ice model (paper Sec. 2: vertical layers of 10 m, each with its
 * own scattering and absorption coefficient).
 *   b_e, a      [n_layers] float32, >= 0: effective scattering and absorption
 *               coefficients (1/m); layer i spans depth
 *               [depth_top_m + i dz_m, depth_top_m + (i + 1) dz_m); depths
 *               outside the table take the nearest edge layer's values
 *   n_layers    1 <= n_layers <= 4096
 *   dz_m        > 0
 *   g           Henyey-Greenstein mean cosine, -1 < g < 1
 * Errors: PP_EINVAL, PP_ENOMEM, PP_ECUDA. */
int pp_load_ice(pp_ctx* ctx, const float* b_e, const float* a, int32_t n_layers,
                float depth_top_m, float dz_m, float g);

/* One event, plain path: one GPU thread per photon, launched for this event
 * alone.  Host buffers.
 *   src[n_src]   sources of the event; photon j of source s has photon id
 *                (sum of n_photons of the sources before s) + j
 *   hits[n_dom]  out: photons that ended on each DOM
 *   counts[4]    out: absorbed (truncated included), escaped, truncated, steps
 * Errors: PP_EINVAL, PP_ENOTLOADED, PP_ECUDA, PP_EDEVICE. */
int pp_propagate(pp_ctx* ctx, uint64_t event_id, const pp_source* src, int64_t n_src,
                 uint64_t* hits, uint64_t* counts);

/* Many events in one persistent launch (cross-event batching, paper Sec. 4:
 * the photon server aggregates steps from many events and clients).  Host
 * buffers.
 *   event_ids[n_events]       event ids (the Philox counter's fourth word, low 32 bits)
 *   src_begin[n_events + 1]   event e owns src[src_begin[e] .. src_begin[e+1]),
 *                             non-decreasing, src_begin[0] = 0
 *   src[src_begin[n_events]]  all sources
 *   hits[n_events][n_dom], counts[n_events][4]  out, as for pp_propagate
 * Errors: PP_EINVAL, PP_ENOTLOADED, PP_ECUDA, PP_EDEVICE. */
int pp_propagate_batch(pp_ctx* ctx, int32_t n_events, const uint64_t* event_ids,
                       const int64_t* src_begin, const pp_source* src, uint64_t* hits,
                       uint64_t* counts);

/* pp_propagate_batch on device-resident inputs and outputs, enqueued on
 * `stream` (NULL: the context's stream); returns once enqueued.
 *   d_event_ids[n_events], d_src_begin[n_events + 1], d_src[n_src] device inputs
 *   n_src                     = src_begin[n_events] (host value)
 *   d_hits[n_events][n_dom], d_counts[n_events][4] device outputs (overwritten)
 * Device errors are latched in the context and returned by pp_sync(). */
int pp_propagate_batch_async(pp_ctx* ctx, int32_t n_events, const uint64_t* d_event_ids,
                             const int64_t* d_src_begin, const pp_source* d_src, int64_t n_src,
                             uint64_t* d_hits, uint64_t* d_counts, void* stream);

/* The plain per-event path on device-resident data: for each event, its own
 * launches with one thread per photon.  Event sizes must be known on the host:
 *   h_event_ids[n_events], h_src_begin[n_events + 1], h_event_photons[n_events]
 *   host arrays; d_src, d_hits, d_counts device buffers as above. */
int pp_propagate_plain_async(pp_ctx* ctx, int32_t n_events, const uint64_t* h_event_ids,
                             const int64_t* h_src_begin, const uint64_t* h_event_photons,
                             const pp_source* d_src, uint64_t* d_hits, uint64_t* d_counts,
                             void* stream);

/* One event on device-resident data with no device allocation during the
 * call.  The paper has no counterpart: this serves callers that may not
 * allocate device memory while they run -- for example a host that hands the
 * library fixed, pre-sized buffers and forbids allocator calls (and the
 * synchronisation cudaMalloc/cudaFree imply) on its hot loop.  The caller
 * passes inputs and outputs as for pp_propagate_batch_async; the kernels'
 * scratch (photon prefix sums, chunk table, work counter) comes from one
 * static device array inside the library, sized for PP_NOALLOC_MAX_SOURCES
 * sources (about 97 KiB, held by every GPU that loads the library until the
 * process exits).
 *   d_src[n_src]  device sources of the event, 0 <= n_src <= PP_NOALLOC_MAX_SOURCES
 *                 (more: PP_EINVAL with a message, nothing enqueued)
 *   d_hits[n_dom], d_counts[4]  device outputs, overwritten (as pp_propagate)
 *   stream        CUDA stream (NULL: the context's stream); returns once enqueued.
 *                 Device errors (a malformed source) are latched in the context
 *                 and returned by pp_sync(ctx, stream) with this same stream,
 *                 which orders the check after this call's kernels.
 * The array's device address is looked up when a context is created on the
 * device (pp_create, with the device current; a context created after a device
 * reset looks it up afresh), so calls need no set-up of their own.  Every
 * call shares the one array and the work
 * counter in it is cleared by each call: calls whose GPU work overlaps in time
 * (different streams, or several contexts on one device) race and must be
 * serialised by the caller.  A call launches two kernels (counted by pp_get_kernel_time). */
#define PP_NOALLOC_MAX_SOURCES 8192
int pp_propagate_noalloc(pp_ctx* ctx, uint64_t event_id, const pp_source* d_src, int64_t n_src,
                         uint64_t* d_hits, uint64_t* d_counts, void* stream);

/* Photons [photon_begin, photon_end) of one event (per-event photon ids, see
 * pp_propagate) through the persistent kernel, on device-resident data.  With
 * accumulate = 0 the outputs are overwritten first, otherwise the tallies are
 * added to them.  Because every photon's random numbers depend only on (seed,
 * event id, photon id), an event split into ranges -- in any order, over any
 * number of calls -- gives exactly the result of one pass: this is how a huge
 * event (paper Sec. 3: power-law energies make single events arbitrarily
 * large) is processed in fixed-size chunks with bounded launch times, and how
 * an interrupted event resumes at its next chunk.
 *   d_src[n_src], d_hits[n_dom], d_counts[4] device buffers; stream as above */
int pp_propagate_range_async(pp_ctx* ctx, uint64_t event_id, const pp_source* d_src,
                             int64_t n_src, uint64_t photon_begin, uint64_t photon_end,
                             int32_t accumulate, uint64_t* d_hits, uint64_t* d_counts,
                             void* stream);

/* ---- compact hit records ------------------------------------------------ */
/* Paper Sec. 4: the hit store keeps only the ID of the particle that
 * produced a hit, the time of the hit and its weight (the diagnostic fields of
 * the older store are dropped).  One record per photon that ends on a DOM:
 *   dom      DOM index (as in hits[])
 *   source   index of the emitting source in the call's d_src array
 *   time_ns  emission offset along the segment at the speed of light plus
 *            the photon's path length at the group velocity c / group_index,
 *            from the segment's start point (sources carry no start time)
 *   weight   the probability that the hit makes a photoelectron (paper Sec. 2:
 *            a function of the photon's position, direction, time and
 *            wavelength, not given there): 1 by default, or the acceptance
 *            polynomial set by pp_set_hit_acceptance.  Hits and counts are
 *            geometric either way. */
typedef struct pp_hit {
  uint32_t dom;
  uint32_t source;
  float time_ns;
  float weight;
} pp_hit;

/* Acceptance of the hit records: weight = clamp(sum_{i < n} coeffs[i] eta^i,
 * 0, 1) with eta the z component of the photon's unit direction when it
 * reaches the DOM (eta = 1: moving straight up, onto the bottom of the DOM).
 * 0 <= n <= PP_MAX_ACCEPT_COEFFS, finite coefficients (host memory, copied);
 * n = 0 restores weight 1.  Errors: PP_EINVAL. */
#define PP_MAX_ACCEPT_COEFFS 8
int pp_set_hit_acceptance(pp_ctx* ctx, const float* coeffs, int32_t n);

/* pp_propagate_batch_async that also writes the hit records: the same hits
 * and counts, plus up to max_records records in d_records[max_records]
 * (device, in no particular order); *d_n_records (device u64, zeroed by the
 * call) receives the number of hits, which may exceed max_records (the excess
 * is counted, not written).  group_index <= 0 selects 1.35; otherwise it must
 * lie in [1, 10).  n_src < 2^32.  Launched directly (never through a cached
 * graph).  Errors: as pp_propagate_batch_async. */
int pp_propagate_records_async(pp_ctx* ctx, int32_t n_events, const uint64_t* d_event_ids,
                               const int64_t* d_src_begin, const pp_source* d_src, int64_t n_src,
                               uint64_t* d_hits, uint64_t* d_counts, float group_index,
                               pp_hit* d_records, uint64_t max_records, uint64_t* d_n_records,
                               void* stream);

/* Waits for `stream` (NULL: the context's stream) and reports a device error
 * flag raised since the last pp_sync.  Errors: PP_ECUDA, PP_EDEVICE. */
int pp_sync(pp_ctx* ctx, void* stream);

/* Launch settings of the persistent kernel (the autotuner's knobs).
 *   block_threads     128, 256, 512 or 1024 (0: keep)
 *   blocks_per_sm     >= 1 (0: as many as fit)
 *   refill_threshold  1..32: a warp gives its idle lanes new photons once at
 *                     least this many of them are idle (0: keep)
 *   photons_per_lane  1: idle lanes are given photons born on the spot, by
 *                     those lanes alone; 2: each warp also keeps up to 48
 *                     photons born ahead in shared memory (2.3 KiB per warp,
 *                     2.6 KiB in the hit-records variant), topped up 32 at a
 *                     time by all of its lanes together, and idle lanes take
 *                     the next of those (0: keep)
 * Defaults: 1024, 0, 2, 2.  Results never depend on these settings (every
 * photon draws its own random numbers and the tallies are integers).
 * Errors: PP_EINVAL. */
int pp_set_launch(pp_ctx* ctx, int32_t block_threads, int32_t blocks_per_sm,
                  int32_t refill_threshold, int32_t photons_per_lane);

/* Autotuner: times the batched path on the given device-resident batch (as
 * pp_propagate_batch_async) for a fixed set of launch settings -- block size
 * 128..1024, 4 to 6 resident 256-thread blocks per SM (register-capped kernel
 * variants), refill thresholds 1..32, one or two photons per lane -- each once
 * untimed and `repeats` times timed with CUDA events on `stream`, keeps the
 * fastest, and reports it in best4 = {block_threads, blocks_per_sm,
 * refill_threshold, photons_per_lane} and best_ms (both may be NULL).  Results
 * do not depend on the settings (the outputs of the last run are valid).
 * Errors: as pp_propagate_batch_async. */
int pp_autotune_batch(pp_ctx* ctx, int32_t n_events, const uint64_t* d_event_ids,
                      const int64_t* d_src_begin, const pp_source* d_src, int64_t n_src,
                      uint64_t* d_hits, uint64_t* d_counts, void* stream, int32_t repeats,
                      int32_t* best4, float* best_ms);

/* Reads back the launch settings in use and the persistent grid they give
 * (any pointer may be NULL). */
int pp_get_launch(const pp_ctx* ctx, int32_t* block_threads, int32_t* blocks_per_sm,
                  int32_t* refill_threshold, int32_t* photons_per_lane, int32_t* grid_blocks);

/* CUDA graphs for pp_propagate_batch_async.  While enabled, the first call with
 * a given shape (event and source counts, device pointers, stream, launch
 * settings) is captured into a CUDA graph -- output clearing, source expansion
 * and the persistent propagation launch -- and later calls with the same shape
 * replay it with one cudaGraphLaunch.  Up to 8 graphs are kept; loading
 * geometry or ice, growing the context's scratch, or disabling graphs drops
 * them.  Calls on the legacy default stream, or with kernel timing enabled,
 * are launched directly. */
int pp_set_graphs(pp_ctx* ctx, int32_t enable);

/* Kernel timing for benchmarks.  While enabled, the library records a pair of
 * CUDA events on the launching stream around every propagation kernel launch.
 * pp_get_kernel_time waits for those events and returns the summed kernel
 * milliseconds and the number of timed launches, plus the number of this
 * library's kernels launched (expansion and propagation, timed or not), all
 * since the previous pp_get_kernel_time; then it resets them. */
int pp_set_kernel_timing(pp_ctx* ctx, int32_t enable);
int pp_get_kernel_time(pp_ctx* ctx, double* total_ms, uint64_t* n_timed, uint64_t* n_kernels);

/* Device memory held by the context's own buffers (tables, scratch, staging;
 * not the surrogate's or a server's), in bytes, and the number of device
 * allocations the context has made since pp_create.  Either pointer may be NULL. */
int pp_get_memory(pp_ctx* ctx, uint64_t* device_bytes, uint64_t* n_allocations);

/* Totals counted by the persistent kernel since the previous call (waits for
 * the device, then resets them): out4 = {steps, layer crossings, photons born,
 * steps that needed the string search of the DOM test}. */
int pp_get_path_stats(pp_ctx* ctx, uint64_t* out4);

/* World cylinder in use: out3 = {radius, z_min, z_max}. */
int pp_get_world(const pp_ctx* ctx, float* out3);

/* ---- serving loop ------------------------------------------------------- */
/* Paper Sec. 4: propagation clients queue photon-emitting steps and send them
 * in blocks to one photon server, which aggregates steps from many events and
 * clients to keep the GPU busy; several client instances share one memory
 * budget.  A pp_server runs that server on a context: any number of host
 * threads submit bunches (pp_submit) and collect their results (pp_collect).
 * Admitted bunches live in a request ring in device memory; a persistent
 * serving kernel claims photons from the ring 32 at a time while requests keep
 * arriving (continuous batching on the device: a bunch admitted while others
 * run is taken by the running kernel, next to them), and raises a flag in
 * host-mapped memory when a bunch's last photon is tallied.  A scheduler
 * thread admits bunches in arrival order while the ring, the device arenas and
 * the budget allow, copies finished bunches' outputs back, and relaunches the
 * kernel.  A launch ends as a whole: idle_exit_us after the server last held
 * unfinished work, or max_launch_ms after it started.  A bunch's result is the
 * same alone and in any mix. */
typedef struct pp_server pp_server; /* opaque */

typedef struct pp_server_config {
  uint64_t budget_bytes;  /* admission cap (default 8 GiB) on the device bytes the
                             admitted bunches occupy: per bunch 40 B per source
                             (arena), 8 B per source + 8 (photon prefix), 4 B per
                             photon chunk + 4 (chunk table), 8 B per DOM + 32
                             (output slot) and 64 B (ring entry).  Photon state
                             lives in registers and shared memory, so no bytes
                             are charged per photon. */
  int64_t arena_sources;  /* device source-arena capacity, also the most sources of
                             one bunch (default 4 194 304) */
  int32_t ring_requests;  /* request-ring slots = bunches admitted at once; a power
                             of two, 1..65536 (default 256) */
  int32_t idle_exit_us;   /* a serving-kernel launch ends once its warps have been
                             idle this long while the server holds no unfinished
                             bunch (default 1000) */
  int32_t max_launch_ms;  /* and stops claiming this long after it started; the
                             scheduler relaunches it (default 200) */
} pp_server_config;

/* Fills *cfg with the defaults above. */
int pp_server_config_default(pp_server_config* cfg);

/* Starts a server on ctx (geometry and ice loaded; while the server exists the
 * context refuses new geometry or ice).  Allocates the ring, the arenas (52 B
 * per arena source), the output slots (8 B per DOM per ring slot) and pinned
 * host mirrors of the same size, and starts the scheduler thread.
 * Errors: PP_EINVAL, PP_ENOTLOADED, PP_ENOMEM. */
int pp_server_create(pp_ctx* ctx, const pp_server_config* cfg, pp_server** out);

/* Runs every submitted bunch to completion, stops the scheduler and frees the
 * server; results not yet collected are discarded. */
int pp_server_destroy(pp_server* server);

/* Message for the last error the server met (never NULL). */
const char* pp_server_last_error(const pp_server* server);

/* Thread-safe.  Copies n_src host sources of one bunch (event id as for
 * pp_propagate) and queues it; *ticket_out identifies it.
 * A bunch with no photons is complete at once (zero outputs).
 * Errors: PP_EINVAL (bad source, 2^35 photons or more), PP_EBUDGET (the bunch
 * alone occupies more than the whole budget, or has more sources than the
 * arena), PP_ECUDA (the server failed earlier). */
int pp_submit(pp_server* server, uint64_t event_id, const pp_source* src, int64_t n_src,
              uint64_t* ticket_out);

/* Thread-safe.  Waits up to timeout_ms (< 0: no limit) for the bunch's result
 * and copies it to hits[n_dom] and counts[4] (either may be NULL); the ticket
 * is then released.  Errors: PP_EINVAL (unknown ticket), PP_ETIMEDOUT (not done
 * yet; the ticket stays valid), PP_EDEVICE / PP_ECUDA (the bunch failed). */
int pp_collect(pp_server* server, uint64_t ticket, uint64_t* hits, uint64_t* counts,
               int32_t timeout_ms);

/* out8 = {bunches done, photons done, p50 latency ms, p99 latency ms,
 * photons/s from first submit to last completion, serving-kernel launches,
 * peak admitted bytes (device bytes occupied by admitted bunches), device
 * bytes the server allocated}; latency = submit to result ready. */
int pp_server_stats(pp_server* server, double* out8);

/* ---- learned surrogate -------------------------------------------------- */
/* No counterpart in the paper's propagation step: an MLP that predicts the
 * expected number of photons a DOM receives from a light source, trained on
 * this library's own Monte Carlo hit counts, so that MC can be replaced where
 * the surrogate is accurate enough and kept as the fallback and as the reference
 * elsewhere.  Network: 32 inputs per (source, DOM) pair -- the ten named
 * (source position, source direction polar/azimuth angles, DOM position
 * relative to the source, effective scattering and absorption at the source's
 * layer) and 22 derived from them and the ice table (unit direction,
 * distance and functions of it, cosine to the DOM, angle and distance from
 * the Cherenkov cone, the ice at the DOM, the mean ice and optical depths
 * along the line to the DOM, DOM height, distance from the track axis) --
 * four hidden layers of 256 SiLU units, output lambda = n_photons *
 * softplus(z).  BF16 weights and activations, FP32 accumulation on the tensor
 * cores (hand-written tcgen05 kernels), FP32 master weights and Adam.
 * Training minimises the Poisson negative log-likelihood mean(lambda - n ln
 * lambda).  Parameters are a flat FP32 array of PP_MLP_N_PARAMS values: W1 [256][32],
 * b1 [256], W2 [256][256], b2, W3, b3, W4, b4, w5 [256], b5 [1] (W[out][in]).
 * An MLP keeps the context's tables in place (like a server); one host thread
 * at a time per MLP; work is enqueued on the context's stream unless a stream
 * is given. */
#define PP_MLP_N_PARAMS 206081
#define PP_MLP_INPUTS 32
typedef struct pp_mlp pp_mlp;

/* Creates a surrogate on ctx (geometry and ice loaded; while it exists the
 * context refuses new geometry or ice).
 *   max_batch  largest training batch, a multiple of 64 (>= 64); training
 *              buffers of ~6 KiB per row are allocated
 *   max_rows   capacity of the inference pair list (8 bytes per row); a
 *              pp_mlp_dom_sums pass holds at most this many pairs
 * Parameters start at zero (use pp_mlp_set_params).
 * Errors: PP_EINVAL, PP_ENOTLOADED, PP_ENOMEM. */
int pp_mlp_create(pp_ctx* ctx, int32_t max_batch, int64_t max_rows, pp_mlp** out);

/* Waits for the device and frees the surrogate.  NULL is accepted. */
int pp_mlp_destroy(pp_mlp* mlp);

/* Message for the last error raised on this surrogate (never NULL). */
const char* pp_mlp_last_error(const pp_mlp* mlp);

/* Host FP32 parameters in / out, n = PP_MLP_N_PARAMS (layout above); set also
 * resets the Adam moments and step.  Both synchronise.
 * Errors: PP_EINVAL (null pointer, wrong n), PP_ECUDA, PP_EDEVICE. */
int pp_mlp_set_params(pp_mlp* mlp, const float* params, int64_t n);
int pp_mlp_get_params(pp_mlp* mlp, float* params, int64_t n);

/* The whole training state, for checkpoint and resume: the FP32 parameters,
 * Adam's first and second moment estimates m and v (Kingma & Ba, "Adam: A
 * Method for Stochastic Optimization", 2015, Algorithm 1), each a host array
 * of n = PP_MLP_N_PARAMS values in the parameter layout above, and the number
 * of Adam steps taken (the next step's bias corrections use step + 1).  get
 * copies out, set copies in (and refreshes the BF16 weight copies).  The moments
 * may be NULL in set (then they start at zero) and in get (not copied); step
 * may be NULL in get.  Both synchronise.
 * Errors: PP_EINVAL (null params, wrong n, step < 0, non-finite values or
 * negative v), PP_ECUDA, PP_EDEVICE. */
int pp_mlp_get_state(pp_mlp* mlp, float* params, float* m, float* v, int64_t n, int64_t* step);
int pp_mlp_set_state(pp_mlp* mlp, const float* params, const float* m, const float* v, int64_t n,
                     int64_t step);

/* Features of n pairs into d_feat[n][32] (BF16 bit patterns, row-major):
 *   d_src              sources as in pp_propagate (the point is the segment's midpoint)
 *   d_pair_src[n], d_pair_dom[n]  indices into d_src and the loaded DOMs (caller-checked)
 * Enqueued on `stream` (NULL: the context's stream).  Errors: PP_EINVAL, PP_ECUDA. */
int pp_mlp_features(pp_mlp* mlp, const pp_source* d_src, const int32_t* d_pair_src,
                    const int32_t* d_pair_dom, int64_t n, uint16_t* d_feat, void* stream);

/* d_lambda[i] = predicted photons on pair i given d_nph[i] photons emitted,
 * by the fused inference kernel (rows mode).  d_feat[n][32] BF16, 16-byte
 * aligned.  Enqueued on `stream` (NULL: the context's stream); a device error
 * (a bounded wait that ran out) is reported by pp_mlp_sync.  The first
 * inference call after the weights change (pp_mlp_set_params, set_state, a
 * train step) reads the hidden biases back to the host, for the kernel's
 * launch parameters, and so waits for `stream` once.
 * Errors: PP_EINVAL (null or misaligned pointer), PP_ECUDA. */
int pp_mlp_forward(pp_mlp* mlp, const uint16_t* d_feat, const float* d_nph, int64_t n,
                   float* d_lambda, void* stream);

/* Forward and backward on one batch without updating: d_feat[n][32] (16-byte
 * aligned), d_nph[n] photons, d_count[n] observed hits; n a multiple of 64 in
 * [64, max_batch].  h_grads[PP_MLP_N_PARAMS] receives d(loss)/d(params) and
 * *h_loss (may be NULL) the mean loss.  Synchronous, on the context's stream.
 * Errors: PP_EINVAL, PP_ECUDA, PP_EDEVICE. */
int pp_mlp_gradients(pp_mlp* mlp, const uint16_t* d_feat, const float* d_nph,
                     const float* d_count, int64_t n, float* h_grads, double* h_loss);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr > 0) on a batch
 * as for pp_mlp_gradients; the batch's mean loss is added to the running sum
 * pp_mlp_loss returns.  Enqueued on `stream` (NULL: the context's stream).
 * Errors: PP_EINVAL, PP_ECUDA (device errors: pp_mlp_sync / pp_mlp_loss). */
int pp_mlp_train_step(pp_mlp* mlp, const uint16_t* d_feat, const float* d_nph,
                      const float* d_count, int64_t n, float lr, void* stream);

/* pp_mlp_train_step on chosen rows of a training set held on the device:
 * d_feat[n_rows][32] (16-byte aligned), d_nph[n_rows], d_count[n_rows] and
 * d_rows[n] (int64 row indices).  One kernel gathers the n rows into the
 * context's batch buffers (an index outside [0, n_rows) raises the device error
 * flag and takes row 0 instead), then the step runs as pp_mlp_train_step.
 * Enqueued on `stream` (NULL: the context's stream).
 * Errors: PP_EINVAL, PP_ECUDA (device errors: pp_mlp_sync / pp_mlp_loss). */
int pp_mlp_train_step_rows(pp_mlp* mlp, const uint16_t* d_feat, const float* d_nph,
                           const float* d_count, int64_t n_rows, const int64_t* d_rows, int64_t n,
                           float lr, void* stream);

/* Sum of the mean losses of the train steps since the last call, then reset.
 * Synchronous.  Errors: PP_EINVAL, PP_ECUDA, PP_EDEVICE. */
int pp_mlp_loss(pp_mlp* mlp, double* loss);

/* Dense inference over n_src sources x all DOMs: d_dom_sums[n_dom] (zeroed
 * here) receives sum over sources of lambda, and d_lambda[n_src][n_dom] (if not
 * NULL, zeroed here) every pair's lambda; d_nph_src[n_src] photons per source.
 * Pairs farther apart than r_max (the distance range the network was trained
 * on) count zero; the pairs within it are found on the device and evaluated
 * by the fused kernel (pairs mode) in passes of at most max_rows pairs.  When
 * n_src x DOMs <= max_rows the call is one pass and returns once it is
 * enqueued on `stream` (NULL: the context's stream); otherwise it enqueues
 * every pass, then waits for the passes' pair counts, and if some pass found
 * more pairs than max_rows it starts over with fewer sources per pass (after
 * the weights change it also waits for the biases, as pp_mlp_forward does).
 * Errors: PP_EINVAL (also: one source with more than max_rows pairs), PP_ECUDA. */
int pp_mlp_dom_sums(pp_mlp* mlp, const pp_source* d_src, int64_t n_src, const float* d_nph_src,
                    float r_max, double* d_dom_sums, float* d_lambda, void* stream);

/* The (source, DOM) pairs closer than r_max (segment midpoint to DOM centre),
 * in (source, DOM) order: the first max_out go to d_pair_src / d_pair_dom, and
 * *h_count receives how many there are (may exceed max_out).  Synchronous, on
 * the context's stream; grows a scratch of 12 bytes per 2048 candidate pairs
 * (n_src x DOMs) when needed.  Errors: PP_EINVAL, PP_ENOMEM, PP_ECUDA. */
int pp_mlp_near_pairs(pp_mlp* mlp, const pp_source* d_src, int64_t n_src, float r_max,
                      int64_t max_out, int32_t* d_pair_src, int32_t* d_pair_dom,
                      uint64_t* h_count);

/* The hidden layers' activation (the network's definition, for training and
 * inference alike; parameters are kept):
 *   PP_MLP_ACT_SILU        silu(z) = z / (1 + exp(-z)) (default)
 *   PP_MLP_ACT_HARD_SWISH  z * clamp(z / 6 + 1/2, 0, 1): no special-function
 *                          operation (the SiLU's one per value caps inference
 *                          at 16 values per SM and clock)
 * Errors: PP_EINVAL. */
#define PP_MLP_ACT_SILU 0
#define PP_MLP_ACT_HARD_SWISH 1
int pp_mlp_set_activation(pp_mlp* mlp, int32_t act);

/* SiLU of the inference kernel: 0 (default) z/2 (1 + tanh.approx(z/2)), one
 * SFU operation per unit; 1: z / (1 + exp(-z)) as in training.  Errors: PP_EINVAL. */
int pp_mlp_set_exact_silu(pp_mlp* mlp, int exact);

/* Waits for the context's stream and reports (then clears) the surrogate's
 * device error flag.  Errors: PP_EINVAL, PP_ECUDA, PP_EDEVICE. */
int pp_mlp_sync(pp_mlp* mlp);

/* ---- debug and parity entry points (host buffers) ------------------------ */

/* Philox4x32-10 blocks computed on the device: out[i] = Philox(ctr[i], key[i]).
 *   ctr[n][4], key[n][2], out[n][4] uint32 */
int pp_debug_philox(pp_ctx* ctx, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                    int64_t n);

/* Follows chosen photons of one event with the production step code and
 * records them.  photon_ids[n] are per-event photon ids.
 *   outcome[n]   out: DOM index, or PP_OUT_ABSORBED / _ESCAPED / _TRUNCATED
 *   n_steps[n]   out: steps taken (Philox blocks drawn after birth)
 *   birth[n][6]  out: birth point and direction (may be NULL)
 *   trace[n][n_trace][3] out: the first n_trace scatter points, NaN after the
 *                photon's last scatter (may be NULL when n_trace = 0) */
int pp_debug_trace(pp_ctx* ctx, uint64_t event_id, const pp_source* src, int64_t n_src,
                   const uint64_t* photon_ids, int64_t n, int32_t n_trace, int32_t* outcome,
                   int64_t* n_steps, float* birth, float* trace);

/* The device scattering step on given directions: the HG polar angle from
 * word x_mu (mapped to u in (0,1) as in the propagation), the azimuth from
 * word x_phi, applied to dir with the context's g.
 *   dir[n][3] unit directions, words[n][2] (x_mu, x_phi), out[n][3] new directions */
int pp_debug_scatter(pp_ctx* ctx, const float* dir, const uint32_t* words, float* out, int64_t n);

/* The tensor-core GEMM of the surrogate on host data: C[M][N] = A[M][K] . B[N][K]^T
 * with A, B BF16 (raw 16-bit patterns, row-major) and C FP32.  16 <= N <= 256,
 * N and K multiples of 16. */
int pp_debug_gemm(pp_ctx* ctx, const uint16_t* A, const uint16_t* B, int32_t M, int32_t N,
                  int32_t K, float* C);

/* The device hit test on given segments: first DOM met on [p, p + S d].
 *   seg[n][7]   p (3), d (3, unit), S
 *   mode        0: string / cell-grid search (production), 1: every DOM
 *   dom[n]      out: DOM index or -1;  t[n] out: distance (inf when none) */
int pp_debug_first_hit(pp_ctx* ctx, const float* seg, int64_t n, int32_t mode, int32_t* dom,
                       float* t);

/* The bounded wait every tensor-core kernel uses for its mbarriers, on one
 * that no arrival completes: it gives up after limit_ns (1e3 .. 1e9) on the
 * global timer and the kernel reports that, so a lost arrival becomes an error
 * status on the host rather than a hung GPU (the kernels then raise their
 * device error flag: PP_EDEVICE from pp_mlp_sync).  One block on `device`.
 *   timed_out  out: 1 if the wait gave up (always, here), 0 if it completed
 *   waited_ns  out: time spent in the wait
 * Errors: PP_EINVAL, PP_ENODEV, PP_ENOMEM, PP_ECUDA. */
int pp_debug_wait_timeout(int32_t device, uint64_t limit_ns, int32_t* timed_out,
                          uint64_t* waited_ns);

/* ---- measured issue rates ------------------------------------------------- */

/* Measured lane-operation rate of one pipe of `device`, the denominator of the
 * propagation kernel's FP32 and SFU utilisation.  A kernel that fills every SM
 * runs independent chains of one instruction per thread, once to warm up and
 * once timed with CUDA events:
 *   PP_ISSUE_FP32_FMA  fmaf chains (one FMA = one lane operation)
 *   PP_ISSUE_SFU_LG2   lg2.approx chains (the special-function unit)
 *   lane_ops_per_s     out: lane operations per second over the whole device
 *   ms                 out: duration of the timed launch (may be NULL)
 * Takes about 0.1 s; allocates 4 bytes and its own stream.  The rate follows
 * the SM clock of the moment.  Errors: PP_EINVAL (unknown kind, NULL output,
 * bad device), PP_ENODEV, PP_ENOMEM, PP_ECUDA. */
#define PP_ISSUE_FP32_FMA 0
#define PP_ISSUE_SFU_LG2 1
int pp_measure_issue_rate(int32_t device, int32_t kind, double* lane_ops_per_s, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* PP_H_ */
