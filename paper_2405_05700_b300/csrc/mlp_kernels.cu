// Kernels of the learned surrogate beside the fused ones (mlp_fused.cu): a
// plain tensor-core GEMM (tcgen05, BF16 in, FP32 accumulate in TMEM) behind
// the debug entry point that checks the operand layout the fused kernels use,
// the pair features and pair search, the head's loss gradient, the ice
// profile's prefix sums, Adam and the BF16 weight copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_internal.h"
#include "mlp_features.cuh"
#include "tc_gemm.cuh"

namespace mlp {

namespace {

constexpr int kBM = 128;      // rows of A / C per CTA (the MMA's M)
constexpr int kBK = 64;       // K staged per round
constexpr uint32_t kWaitTries = 1u << 22;

__device__ __forceinline__ uint32_t pow2_cols(int n) {
  return n > 128 ? 256u : (n > 64 ? 128u : (n > 32 ? 64u : 32u));
}

// Copies rows [r0, r0 + rows) x K columns [k0, k0 + kBK) of a row-major BF16
// matrix (leading dimension ld) into a K-major no-swizzle smem tile; rows or
// columns outside (n_rows, K) are zero.  Four 16-byte loads are in flight per
// thread before their stores.
__device__ __forceinline__ void stage_tile(unsigned char* tile, const __nv_bfloat16* X, int ld,
                                           int n_rows, int K, int r0, int rows, int k0) {
  const int chunks = rows * (kBK / 8);
  const int step = blockDim.x;
  for (int base = threadIdx.x; base < chunks; base += 4 * step) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * step;
      const int r = i >> 3, c = i & 7;
      const int gr = r0 + r, gk = k0 + c * 8;
      v[u] = make_uint4(0, 0, 0, 0);
      if (i < chunks && gr < n_rows && gk < K)
        v[u] = *reinterpret_cast<const uint4*>(X + (size_t)gr * ld + gk);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = base + u * step;
      if (i < chunks)
        *reinterpret_cast<uint4*>(tile + tc::tile_off(i >> 3, (i & 7) * 8, kBK)) = v[u];
    }
  }
}

// Two operand stages: while the tensor core works on one, the threads stage
// the next K slice into the other.
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t bar[2];
  const int BN = g.bn;
  const int stage = (kBM + BN) * kBK * 2;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kb = 0, ke = g.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = pow2_cols(BN);
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  const uint32_t idesc = tc::idesc_bf16(kBM, BN);
  // descriptor strides: K-direction core matrices 128 B apart, 8-row groups
  // kBK * 16 B apart (exchanged when probing the layout)
  const uint32_t lbo = 128, sbo = kBK * 16;  // K-direction and row-direction core-matrix strides
  uint32_t phase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  int it = 0;
  for (int k0 = kb; k0 < ke; k0 += kBK, ++it) {
    const int b = it & 1;
    if (pending[b]) {  // the MMAs that read this stage two rounds ago must be done
      const bool done = tc::mbar_wait(&bar[b], phase[b], kWaitTries);
      phase[b] ^= 1u;
      pending[b] = false;
      ok = __syncthreads_and(done);
      if (!ok) break;
    }
    unsigned char* sA = smem + b * stage;
    unsigned char* sB = sA + kBM * kBK * 2;
    stage_tile(sA, g.A, g.lda, g.M, ke, m0, kBM, k0);
    stage_tile(sB, g.B, g.ldb, g.N, ke, n0, BN, k0);
    tc::fence_smem_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s) {
        if (k0 + 16 * s >= ke) break;
        tc::mma_bf16(taddr, tc::smem_desc(a0 + 256 * s, lbo, sbo),
                     tc::smem_desc(b0 + 256 * s, lbo, sbo), idesc, (k0 > kb || s > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[b]);
    }
    pending[b] = true;
  }
  // drain the stages still in flight (MMAs complete in issue order)
  for (int b = 0; b < 2; ++b) {
    if (!pending[b]) continue;
    const bool done = tc::mbar_wait(&bar[b], phase[b], kWaitTries);
    phase[b] ^= 1u;
    ok = __syncthreads_and(done && ok);
  }
  tc::fence_after_sync();
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(g.err, 1);
  } else if (kb < ke) {
    // epilogue: warp w owns rows m0 + 32 w + lane; 32 columns per TMEM load
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = n0 + c0 + j;
        if (col >= g.N || c0 + j >= BN) continue;
        g.Cf[(size_t)row * g.ldc + col] = v[j];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

}  // namespace

size_t gemm_smem_bytes(int bn) { return 2 * (size_t)(kBM + bn) * kBK * 2 + 1024; }

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  const dim3 grid((g.M + kBM - 1) / kBM, (g.N + g.bn - 1) / g.bn);
  const size_t smem = gemm_smem_bytes(g.bn);
  // at least 80 KB per CTA: at most two CTAs (2 x 256 TMEM columns) per SM
  const size_t smem_req = smem < 80 * 1024 ? 80 * 1024 : smem;
  cudaError_t e = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_req);
  if (e != cudaSuccess) return e;
  k_gemm<<<grid, 128, smem_req, st>>>(g);
  return cudaGetLastError();
}

// ------------------------------------------------------------- features --
namespace {

__global__ void k_ice_cum(FeatGeom fg, float2* cum) {
  double sb = 0.0, sa = 0.0;
  for (int i = 0; i < fg.L; ++i) {
    cum[i] = make_float2((float)sb, (float)sa);
    const float4 l = fg.layer[i];
    sb += (double)(l.x * fg.be_over_b);
    sa += (double)l.y;
  }
}

__global__ void k_features(FeatGeom fg, const pp_source* src, const int32_t* ps, const int32_t* pd,
                           int64_t n, __nv_bfloat16* feat) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  pair_features(fg, src[ps[i]], fg.dom[pd[i]], feat + i * kIn);
}

// ------------------------------------------------------------------ head --
__device__ __forceinline__ float softplus(float z) { return z > 20.0f ? z : log1pf(__expf(z)); }

// z of pair p by one warp: 256 BF16 activations . w5
__device__ __forceinline__ float head_z(const __nv_bfloat16* hp, const float* w5, float b5) {
  const int lane = threadIdx.x & 31;
  const uint4 raw = *reinterpret_cast<const uint4*>(hp + lane * 8);
  const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&raw);
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc = fmaf(__bfloat162float(hv[j]), w5[lane * 8 + j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc + b5;
}

constexpr int kHeadPairs = kHeadPartPairs;  // pairs per block of the head backward
constexpr int kHeadCols = kHeadPartCols;    // W5 and b5: one partial-sum row per block
static_assert(kHeadCols == kHid + 1, "W5 and b5");

// Head backward on a block of kHeadPairs pairs: dz4, and the block's partial
// sums of dL/dW5, dL/db5 (part[block][257]) and of the loss (lpart[block]).
// Every sum runs in a fixed order, so the gradients do not depend on timing.
__global__ void __launch_bounds__(256) k_head_bwd(const __nv_bfloat16* h, const __nv_bfloat16* z4,
                                                  const float* w5, const float* b5,
                                                  const float* nph, const float* cnt, int64_t n,
                                                  float inv_n, __nv_bfloat16* dz4, float* part,
                                                  double* lpart, int act) {
  __shared__ float s_g[kHeadPairs];
  __shared__ float s_w5[kHid];
  __shared__ float s_gsum[8];
  __shared__ double s_lsum[8];
  const int64_t p0 = (int64_t)blockIdx.x * kHeadPairs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  s_w5[threadIdx.x] = w5[threadIdx.x];
  __syncthreads();
  double lsum = 0.0;
  float gsum = 0.0f;
  for (int q = warp; q < kHeadPairs; q += 8) {
    const int64_t p = p0 + q;
    float g = 0.0f;
    if (p < n) {
      const float z = head_z(h + p * kHid, s_w5, *b5);
      const float sp = fmaxf(softplus(z), 1e-30f);
      const float lam = nph[p] * sp;
      const float k = cnt[p];
      const float sig = 1.0f / (1.0f + __expf(-z));
      g = nph[p] * sig * (1.0f - k / lam) * inv_n;
      if (lane == 0) lsum += (double)(lam - (k > 0.0f ? k * logf(lam) : 0.0f)) * inv_n;
    }
    if (lane == 0) {
      s_g[q] = g;
      gsum += g;
    }
  }
  if (lane == 0) {
    s_gsum[warp] = gsum;
    s_lsum[warp] = lsum;
  }
  __syncthreads();
  const int j = threadIdx.x;
  float acc = 0.0f;
  for (int q = 0; q < kHeadPairs; ++q) {
    const int64_t p = p0 + q;
    if (p >= n) break;
    const float g = s_g[q];
    const size_t o = (size_t)p * kHid + j;
    acc = fmaf(g, __bfloat162float(h[o]), acc);
    dz4[o] = __float2bfloat16_rn(g * s_w5[j] * act_grad(act, __bfloat162float(z4[o])));
  }
  float* row = part + (size_t)blockIdx.x * kHeadCols;
  row[j] = acc;
  if (j == 0) {
    float gs = 0.0f;
    double ls = 0.0;
    for (int w = 0; w < 8; ++w) {
      gs += s_gsum[w];
      ls += s_lsum[w];
    }
    row[kHid] = gs;
    lpart[blockIdx.x] = ls;
  }
}

// dW5, db5 (257 values) += the column sums of part[parts][257]; *loss += the
// sum of lpart[parts].  Blocks 0..8 take 32 columns each: warp w sums rows
// w, w + 8, ..., and the eight warp sums are added in warp order.  Block 9
// sums the loss partials the same way (256 threads, then lanes and warps in a
// fixed tree).  Every sum has a fixed order: the result does not depend on
// timing.
constexpr int kHeadReduceColBlocks = (kHeadCols + 31) / 32;

__global__ void __launch_bounds__(256) k_head_reduce(const float* part, const double* lpart,
                                                     int parts, float* dw5b5, double* loss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (blockIdx.x < kHeadReduceColBlocks) {
    __shared__ float ws[8][32];
    const int col = blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (col < kHeadCols) {
#pragma unroll 8
      for (int c = warp; c < parts; c += 8) acc += part[(size_t)c * kHeadCols + col];
    }
    ws[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && col < kHeadCols) {
      float t = 0.0f;
      for (int w = 0; w < 8; ++w) t += ws[w][lane];
      dw5b5[col] += t;
    }
  } else {
    __shared__ double wl[8];
    double acc = 0.0;
    for (int c = threadIdx.x; c < parts; c += 256) acc += lpart[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wl[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += wl[w];
      *loss += t;
    }
  }
}

// Is candidate i = (source s0 + i / n_dom, DOM i % n_dom) within r_max?  The
// distance is from the segment's midpoint to the DOM centre, as in the
// features; the test compares squares (no square root or division per pair).
__device__ __forceinline__ bool pair_near(const FeatGeom& fg, const pp_source* src, int64_t s0,
                                          int64_t i, float r_max, int64_t& s, int& d) {
  s = s0 + i / fg.n_dom;
  d = (int)(i % fg.n_dom);
  const pp_source q = src[s];
  const float nn = fmaf(q.dx, q.dx, fmaf(q.dy, q.dy, q.dz * q.dz));
  const float h = nn > 0.0f ? 0.5f * q.length * rsqrtf(nn) : 0.0f;  // half length / |d|
  const float4 c = fg.dom[d];
  const float ex = c.x - fmaf(h, q.dx, q.x), ey = c.y - fmaf(h, q.dy, q.y),
              ez = c.z - fmaf(h, q.dz, q.z);
  return fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= r_max * r_max;
}

// Pairs of sources [s0, s0 + ns) x all DOMs within r_max, appended in any
// order (one atomic per warp); at most max_out are written, *count counts
// them all.  The per-DOM sums of the inference do not depend on the order.
__global__ void k_near_pairs(FeatGeom fg, const pp_source* src, int64_t s0, int64_t ns,
                             float r_max, int64_t max_out, int32_t* ps, int32_t* pd,
                             unsigned long long* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool near = false;
  int64_t s = 0;
  int d = 0;
  if (i < ns * fg.n_dom) near = pair_near(fg, src, s0, i, r_max, s, d);
  const unsigned mask = __ballot_sync(0xffffffffu, near);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == __ffs(mask) - 1) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
  if (near) {
    const unsigned long long o = base + __popc(mask & ((1u << lane) - 1u));
    if ((int64_t)o < max_out) {
      ps[o] = (int32_t)s;
      pd[o] = d;
    }
  }
}

// The same list in (source, DOM) order: a stable compaction in three passes.
// A block covers kNearTile consecutive candidates, kNearItems per thread.
constexpr int kNearThreads = 256;
constexpr int kNearItems = 8;
constexpr int kNearTile = kNearThreads * kNearItems;
constexpr int kNearScanThreads = 1024;

// Bit j of the result: candidate first + j is a pair within r_max.
__device__ __forceinline__ uint32_t near_bits(const FeatGeom& fg, const pp_source* src, int64_t s0,
                                              int64_t first, int64_t total, float r_max) {
  uint32_t bits = 0;
#pragma unroll
  for (int j = 0; j < kNearItems; ++j) {
    const int64_t i = first + j;
    int64_t s;
    int d;
    if (i < total && pair_near(fg, src, s0, i, r_max, s, d)) bits |= 1u << j;
  }
  return bits;
}

// Exclusive prefix of v over the block's threads (256); *total = the sum.
__device__ __forceinline__ uint32_t block_excl_256(uint32_t v, uint32_t* ws, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  uint32_t before = 0;
  total = 0;
  for (int w = 0; w < kNearThreads / 32; ++w) {
    if (w < warp) before += ws[w];
    total += ws[w];
  }
  return before + x - v;
}

__global__ void __launch_bounds__(kNearThreads) k_near_count(FeatGeom fg, const pp_source* src,
                                                             int64_t s0, int64_t total,
                                                             float r_max, uint32_t* bcount) {
  __shared__ uint32_t ws[kNearThreads / 32];
  const int64_t first = (int64_t)blockIdx.x * kNearTile + (int64_t)threadIdx.x * kNearItems;
  const uint32_t c = __popc(near_bits(fg, src, s0, first, total, r_max));
  uint32_t sum;
  block_excl_256(c, ws, sum);
  if (threadIdx.x == 0) bcount[blockIdx.x] = sum;
}

// One block: boff[b] = sum of bcount[0..b), *count = the sum of all.
__global__ void __launch_bounds__(kNearScanThreads) k_near_scan(const uint32_t* bcount, int64_t nb,
                                                                unsigned long long* boff,
                                                                unsigned long long* count) {
  __shared__ unsigned long long ws[kNearScanThreads];
  const int t = threadIdx.x;
  const int64_t seg = (nb + kNearScanThreads - 1) / kNearScanThreads;
  const int64_t b0 = t * seg, b1 = b0 + seg < nb ? b0 + seg : nb;
  unsigned long long mine = 0;
  for (int64_t b = b0; b < b1; ++b) mine += bcount[b];
  ws[t] = mine;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 segment sums
  for (int o = 1; o < kNearScanThreads; o <<= 1) {
    const unsigned long long y = t >= o ? ws[t - o] : 0ull;
    __syncthreads();
    ws[t] += y;
    __syncthreads();
  }
  unsigned long long run = ws[t] - mine;
  for (int64_t b = b0; b < b1; ++b) {
    boff[b] = run;
    run += bcount[b];
  }
  if (t == kNearScanThreads - 1) *count = ws[t];
}

__global__ void __launch_bounds__(kNearThreads) k_near_write(FeatGeom fg, const pp_source* src,
                                                             int64_t s0, int64_t total,
                                                             float r_max,
                                                             const unsigned long long* boff,
                                                             int64_t max_out, int32_t* ps,
                                                             int32_t* pd) {
  __shared__ uint32_t ws[kNearThreads / 32];
  const int64_t first = (int64_t)blockIdx.x * kNearTile + (int64_t)threadIdx.x * kNearItems;
  uint32_t bits = near_bits(fg, src, s0, first, total, r_max);
  uint32_t sum;
  unsigned long long o = boff[blockIdx.x] + block_excl_256(__popc(bits), ws, sum);
  while (bits) {
    const int j = __ffs(bits) - 1;
    bits &= bits - 1;
    if ((int64_t)o < max_out) {
      ps[o] = (int32_t)(s0 + (first + j) / fg.n_dom);
      pd[o] = (int32_t)((first + j) % fg.n_dom);
    }
    ++o;
  }
}

// Training batch from chosen rows: out[i] = in[rows[i]] for the 64-byte
// feature rows, photons and counts.  A row index outside [0, n_rows) raises
// the error flag and reads row 0.
__global__ void k_gather_rows(const uint4* feat, const float* nph, const float* cnt, int64_t n_rows,
                              const int64_t* rows, int64_t n, uint4* feat_out, float* nph_out,
                              float* cnt_out, int* err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one 16-byte part
  if (t >= n * 4) return;
  const int64_t i = t >> 2;
  int64_t r = rows[i];
  if (r < 0 || r >= n_rows) {
    atomicOr(err, kGatherBadRow);
    r = 0;
  }
  feat_out[t] = feat[r * 4 + (t & 3)];
  if ((t & 3) == 0) {
    nph_out[i] = nph[r];
    cnt_out[i] = cnt[r];
  }
}

__global__ void k_src_prep(FeatGeom fg, const pp_source* src, int64_t s0, int64_t ns,
                           SrcPrep* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) out[i] = source_prep(fg, src[s0 + i]);
}

// ----------------------------------------------------------- utilities --
__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                       float b2, float eps, float bc1, float bc2, __nv_bfloat16* pb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  p[i] = pi;
  if (pb) pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* in, int64_t n, __nv_bfloat16* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_ice_cum(const FeatGeom& fg, float2* cum, cudaStream_t st) {
  k_ice_cum<<<1, 1, 0, st>>>(fg, cum);
  return cudaGetLastError();
}

cudaError_t launch_features(const FeatGeom& fg, const pp_source* src, const int32_t* pair_src,
                            const int32_t* pair_dom, int64_t n, __nv_bfloat16* feat,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_features<<<blocks_for(n, 256), 256, 0, st>>>(fg, src, pair_src, pair_dom, n, feat);
  return cudaGetLastError();
}

cudaError_t launch_head_backward(const __nv_bfloat16* h, const __nv_bfloat16* z4, const float* w5,
                                 const float* b5, const float* nph, const float* cnt, int64_t n,
                                 float inv_n, __nv_bfloat16* dz4, float* dw5b5, double* loss,
                                 float* part, double* lpart, int64_t part_rows, int act,
                                 cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + kHeadPairs - 1) / kHeadPairs;
  if (blocks > part_rows) return cudaErrorInvalidValue;
  k_head_bwd<<<(unsigned)blocks, 256, 0, st>>>(h, z4, w5, b5, nph, cnt, n, inv_n, dz4, part, lpart,
                                               act);
  k_head_reduce<<<kHeadReduceColBlocks + 1, 256, 0, st>>>(part, lpart, (int)blocks, dw5b5, loss);
  return cudaGetLastError();
}

cudaError_t launch_near_pairs(const FeatGeom& fg, const pp_source* src, int64_t s0, int64_t ns,
                              float r_max, int64_t max_out, int32_t* ps, int32_t* pd,
                              unsigned long long* count, cudaStream_t st) {
  const int64_t n = ns * fg.n_dom;
  if (n <= 0) return cudaSuccess;
  k_near_pairs<<<blocks_for(n, 256), 256, 0, st>>>(fg, src, s0, ns, r_max, max_out, ps, pd, count);
  return cudaGetLastError();
}

int64_t near_pairs_ordered_blocks(int64_t n_candidates) {
  return (n_candidates + kNearTile - 1) / kNearTile;
}

cudaError_t launch_near_pairs_ordered(const FeatGeom& fg, const pp_source* src, int64_t ns,
                                      float r_max, int64_t max_out, int32_t* ps, int32_t* pd,
                                      unsigned long long* count, uint32_t* bcount,
                                      unsigned long long* boff, cudaStream_t st) {
  const int64_t n = ns * fg.n_dom;
  if (n <= 0) return cudaSuccess;
  const int64_t nb = near_pairs_ordered_blocks(n);
  if (nb > 0x7fffffff) return cudaErrorInvalidValue;
  k_near_count<<<(unsigned)nb, kNearThreads, 0, st>>>(fg, src, 0, n, r_max, bcount);
  k_near_scan<<<1, kNearScanThreads, 0, st>>>(bcount, nb, boff, count);
  k_near_write<<<(unsigned)nb, kNearThreads, 0, st>>>(fg, src, 0, n, r_max, boff, max_out, ps, pd);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, __nv_bfloat16* pb,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_adam<<<blocks_for(n, 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, pb);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const __nv_bfloat16* feat, const float* nph, const float* cnt,
                               int64_t n_rows, const int64_t* rows, int64_t n,
                               __nv_bfloat16* feat_out, float* nph_out, float* cnt_out, int* err,
                               cudaStream_t st) {
  static_assert(kIn * 2 == 4 * 16, "a feature row is four 16-byte parts");
  if (n <= 0) return cudaSuccess;
  k_gather_rows<<<blocks_for(n * 4, 256), 256, 0, st>>>(
      reinterpret_cast<const uint4*>(feat), nph, cnt, n_rows, rows, n,
      reinterpret_cast<uint4*>(feat_out), nph_out, cnt_out, err);
  return cudaGetLastError();
}

cudaError_t launch_src_prep(const FeatGeom& fg, const pp_source* src, int64_t s0, int64_t ns,
                            SrcPrep* out, cudaStream_t st) {
  if (ns <= 0) return cudaSuccess;
  k_src_prep<<<blocks_for(ns, 256), 256, 0, st>>>(fg, src, s0, ns, out);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* in, int64_t n, __nv_bfloat16* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_to_bf16<<<blocks_for(n, 256), 256, 0, st>>>(in, n, out);
  return cudaGetLastError();
}

}  // namespace mlp
