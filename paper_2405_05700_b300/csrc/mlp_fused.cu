// Fused surrogate inference: features, the four hidden layers and the Poisson
// head of 256 pairs per tile in one persistent kernel, the activations never
// leaving the SM.
//
// Per CTA (one per SM): two row halves of 128 pairs, each an M = 128 tcgen05
// MMA chain with its FP32 accumulator (256 columns) in TMEM.  The halves run
// in ping-pong: while the tensor core computes one half's layer, the other
// half's epilogue converts its previous layer, so MMAs and epilogues overlap.
// A layer's input (features, then BF16 activations) sits in shared memory as
// the MMA's A operand; the weights (W1 as one 16 KB chunk, then 4 chunks of
// 32 KB per hidden layer) stream from global memory (L2-resident, shared by
// every CTA) through a 3-stage ring filled by bulk copies, once per half.
// Each chunk costs a fixed round trip (its MMAs' commit frees the stage, the
// producer's copy refills it), so the ring holds few large chunks: 32 KB
// chunks in 2 stages run the kernel 13 % faster than 16 KB ones in 5 stages
// (8 KB ones in 10 stages are 65 % slower), and a third 32 KB stage another
// 7 %.  The third stage takes the shared memory of the halved biases, which
// inference passes as a launch parameter (read through the constant cache;
// the training forward keeps them in shared memory and two stages).
//
//   warps 0-15 : epilogue.  Warp w serves half (w / 4) % 2, TMEM lanes
//                32 (w % 4) .. + 31 (its 32 rows) and columns 128 (w / 8) .. + 127:
//                features (column group 0), bias + SiLU to BF16 back into shared
//                memory, the head (the two column groups' partial dot products
//                meet in shared memory)
//   warp 16    : producer of the weight ring
//   warp 17    : MMA issue (one thread)
//
// Every wait is bounded; a wait that runs out raises the CTA's abort flag and
// the device error flag, and every role then leaves its loop.
#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_features.cuh"
#include "mlp_internal.h"
#include "tc_gemm.cuh"

namespace mlp {

namespace {

constexpr int kRows = 256;                 // pairs per tile
constexpr int kHalf = 128;                 // rows per MMA
constexpr int kChunkK = 64;                // K per weight chunk of a hidden layer
constexpr int kChunksPerLayer = kHid / kChunkK;
constexpr int kChunkBytes = kHid * kChunkK * 2;
// weight-ring stages: three 32 KB chunks in flight for inference and for the
// backward pass; two for the training forward, whose halved biases take
// shared memory (inference reads them from its launch parameter)
constexpr int kStagesMax = 3;
constexpr int kW1Bytes = kHid * kIn * 2;   // W1: one chunk of K = kIn
constexpr int kHiddenGemms = kLayers - 1;  // layers 2..4
constexpr int kChunksPerLayerSet = 1 + kHiddenGemms * kChunksPerLayer;  // W1..W4
constexpr int kChunksPerTile = 2 * kChunksPerLayerSet;                   // once per half
static_assert(kIn <= kChunkK && kIn % 16 == 0, "W1 is one ring chunk");
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = kEpiThreads + 64;
constexpr int kProducerWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kColsPerWarp = kHid / 2;
// columns per TMEM load in the forward epilogue: 16 (two register sets of 16
// leave the compiler room to overlap the conversions; 32 were 1.4 % slower)
constexpr int kEpiCols = 16;
// 18 warps: two of the four schedulers hold 5 warps, whose registers come from
// that scheduler's 16K, so a thread gets at most 96 registers
constexpr uint32_t kWaitTries = 1u << 22;

// dynamic shared memory
constexpr uint32_t kOffH = 0;                                  // 2 x [128][256] BF16 (features alias)
constexpr uint32_t kHalfBytes = kHalf * kHid * 2;
constexpr uint32_t kOffRing = kOffH + 2 * kHalfBytes;
template <bool kTrain>
struct FwdLayout {
  static constexpr int kStages = kTrain ? 2 : kStagesMax;
  // FP32 parameters after the ring: training: biases / 2 [4][256], then w5
  // [256]; inference: w5 only
  static constexpr uint32_t kOffPar = kOffRing + kStages * kChunkBytes;
  static constexpr uint32_t kW5 = kTrain ? kLayers * kHid : 0;  // w5's offset in floats
  static constexpr uint32_t kSmemBytes = kOffPar + (kW5 + kHid) * 4;
};
// 2 KB of static shared memory (barriers, the head's partial sums) besides
static_assert(FwdLayout<false>::kSmemBytes + 2048 <= 232448 &&
                  FwdLayout<true>::kSmemBytes + 2048 <= 232448,
              "shared memory per CTA");
constexpr int kBwdStages = kStagesMax;
constexpr uint32_t kBwdSmemBytes = kOffRing + kBwdStages * kChunkBytes;
static_assert(kBwdSmemBytes + 1024 <= 232448, "shared memory per CTA");

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// silu(z) = z sigmoid(z) = h (1 + tanh h) with h = z / 2: one SFU operation
// (the epilogue evaluates h tanh h + h with ffma2, two columns at a time).

__device__ __forceinline__ float softplus(float z) { return z > 20.0f ? z : log1pf(__expf(z)); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float silu_exact(float z) { return z / (1.0f + __expf(-z)); }

// Two FP32 fused multiply-adds in one instruction (PTX fma.rn.f32x2, sm_100 and
// later): d.x = a.x b.x + c.x, d.y = a.y b.y + c.y, each rounded to nearest as
// fmaf is, so the results are those of two fmaf calls.  The epilogue issues
// half as many FMA instructions, which leaves more issue slots on its
// schedulers to the producer and MMA threads of the weight ring.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

__device__ __forceinline__ void epi_ld(uint32_t taddr, uint32_t (&r)[16]) { tc::tmem_ld16_nowait(taddr, r); }

// kTrain: rows mode for training -- also writes each layer's BF16
// pre-activations (row-major [n][256]) and activations (the first three
// layers transposed, [256][n], as the weight-gradient GEMMs read them; the
// last row-major, for the head) to global memory.
// kMode: how the hidden-layer activation is evaluated
//   kModeSiluFast   silu(z) = h (1 + tanh h), h = z / 2: one tanh.approx
//   kModeSiluExact  z / (1 + exp(-z))
//   kModeHardSwish  z * clamp(z / 6 + 1/2, 0, 1): FMA pipe only
constexpr int kModeSiluFast = 0, kModeSiluExact = 1, kModeHardSwish = 2;
template <bool kFromPairs, int kMode, bool kTrain = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_fused(FusedArgs a, const __grid_constant__ HalfBias hbias_par) {
  using L = FwdLayout<kTrain>;
  constexpr int kStages = L::kStages;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], in_ready[2], done;
  __shared__ __align__(8) uint64_t head_bar[8];  // per (half, lane quarter): partial z written
  __shared__ float zpart[kRows];                 // column group 1's partial head sums
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // rows: a.n, or the pair search's count in device memory capped at a.n
  // (read here, so that the host need not wait for it)
  const int64_t n_rows = a.n_dev ? (int64_t)min((unsigned long long)a.n, *a.n_dev) : a.n;
  const int64_t n_tiles = (n_rows + kRows - 1) / kRows;

  // setup: TMEM (512 columns: both accumulators), barriers, resident parameters
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int h = 0; h < 2; ++h) {
      tc::mbar_init(&acc_full[h], 1);
      tc::mbar_init(&in_ready[h], kEpiThreads / 2);
    }
    tc::mbar_init(&done, 1);
    for (int i = 0; i < 8; ++i) tc::mbar_init(&head_bar[i], 32);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    // halved biases: the epilogue forms z / 2 = acc / 2 + b / 2 in one FMA
    // (inference: hbias_par holds them already)
    float* par = reinterpret_cast<float*>(smem + L::kOffPar);
    if (kTrain)
      for (int i = threadIdx.x; i < kLayers * kHid; i += blockDim.x)
        par[i] = 0.5f * a.bias[i / kHid][i % kHid];
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) par[L::kW5 + i] = a.w5[i];
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------- producer --
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int jt = 0; jt < kChunksPerTile; ++jt, ++it) {
          // job order (layer, half); the packed image holds W1 (kW1Bytes), then
          // hidden layer l's chunk c at kW1Bytes + (4 (l - 1) + c) kChunkBytes
          const int layer = jt < 2 ? 0 : 1 + (jt - 2) / (2 * kChunksPerLayer);
          const int c = jt < 2 ? 0 : (jt - 2) % kChunksPerLayer;
          const uint32_t s = it % kStages;
          if (it >= (uint32_t)kStages) {
            if (!tc::mbar_wait(&empty[s], ((it / kStages) - 1) & 1, kWaitTries) ||
                *(volatile int*)&abort_flag) {
              ok = false;
              break;
            }
          }
          const uint32_t bytes = layer == 0 ? (uint32_t)kW1Bytes : (uint32_t)kChunkBytes;
          const size_t src =
              layer == 0 ? 0
                         : (size_t)kW1Bytes +
                               (size_t)((layer - 1) * kChunksPerLayer + c) * kChunkBytes;
          tc::mbar_arrive_expect_tx(&full[s], bytes);
          tc::bulk_g2s(smem + kOffRing + s * kChunkBytes, a.wpack + src, bytes, &full[s]);
        }
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        atomicOr(a.err, 1);
      }
      // the copies this thread started have landed before the CTA may exit
      const uint32_t last = it < (uint32_t)kStages ? it : (uint32_t)kStages;
      for (uint32_t q = 0; q < last; ++q) {
        const uint32_t i = it - 1 - q;
        tc::mbar_wait(&full[i % kStages], (i / kStages) & 1, kWaitTries);
      }
    }
  } else if (warp == kMmaWarp) {
    // --------------------------------------------------------------- MMA --
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kHalf, kHid);
      const uint32_t sh = tc::smem_u32(smem + kOffH);
      const uint32_t ring = tc::smem_u32(smem + kOffRing);
      uint32_t it = 0, in_phase[2] = {0u, 0u};
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        // jobs (layer, half) in order: half h's layer l waits for its own
        // epilogue of layer l - 1, which overlaps the other half's MMAs
        for (int job = 0; job < 2 * kLayers && ok; ++job) {
          const int layer = job >> 1, h = job & 1;
          if (!tc::mbar_wait(&in_ready[h], in_phase[h] & 1, kWaitTries) ||
              *(volatile int*)&abort_flag) {
            ok = false;
            break;
          }
          ++in_phase[h];
          tc::fence_after_sync();
          // layer 0: features (32 columns) x W1 (one chunk); then 4 chunks per layer
          const int chunks = layer == 0 ? 1 : kChunksPerLayer;
          const uint32_t sbo_a = (layer == 0 ? kIn : kHid) * 16;
          for (int c = 0; c < chunks; ++c, ++it) {
            const uint32_t s = it % kStages;
            if (!tc::mbar_wait(&full[s], (it / kStages) & 1, kWaitTries)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t b0 = ring + s * kChunkBytes;
            const int kc = layer == 0 ? kIn : kChunkK;  // K of this chunk
#pragma unroll
            for (int kk = 0; kk < kChunkK / 16; ++kk) {
              if (kk * 16 < kc) {
                const uint32_t k0 = c * kChunkK + kk * 16;
                tc::mma_bf16(tmem + h * kHid,
                             tc::smem_desc(sh + h * kHalfBytes + k0 * 16, 128, sbo_a),
                             tc::smem_desc(b0 + kk * 256, 128, kc * 16), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
              }
            }
            tc::mma_commit(&empty[s]);
          }
          tc::mma_commit(&acc_full[h]);
        }
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        atomicOr(a.err, 1);
      }
      // every MMA issued here has completed before TMEM is released
      tc::mma_commit(&done);
      tc::mbar_wait(&done, 0, kWaitTries);
    }
  } else {
    // ---------------------------------------------------------- epilogue --
    const int q = warp & 3, h = (warp >> 2) & 1, cg = warp >> 3;
    const int r = q * 32 + lane;  // row within the half = TMEM lane
    const int c_begin = cg * kColsPerWarp;
    unsigned char* sH = smem + kOffH + h * kHalfBytes;
    const float* par = reinterpret_cast<const float*>(smem + L::kOffPar);
    const uint32_t tacc =
        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * kHid) + (uint32_t)c_begin;
    uint64_t* hb = &head_bar[h * 4 + q];
    uint32_t acc_phase = 0, head_phase = 0;
    bool ok = true;
    // The features of a tile's rows are the first MMA's A operand (aliasing
    // the activations).  Each thread gathers its row's part into registers
    // (pairs: column group g computes features 16 g .. 16 g + 15; rows: column
    // group 0 loads all 32) and stores them once the half's shared memory is
    // free.  For the next tile that happens while the last layer's MMAs run:
    // the gather's loads or arithmetic overlap them, the store follows the
    // last accumulator's arrival (its MMAs no longer read the activations),
    // and the half's next first-layer MMA may start as soon as the last
    // layer's accumulator has been read (a fifth of the tile's time went to
    // the feature gather between tiles before).
    constexpr int kFeatVecs = kFromPairs ? kIn / 16 : kIn / 8;
    uint4 fv[kFeatVecs];
    auto gather_features = [&](int64_t tt) {
      const int64_t frow = tt * kRows + h * kHalf + r;
#pragma unroll
      for (int i = 0; i < kFeatVecs; ++i) fv[i] = make_uint4(0, 0, 0, 0);
      if (frow >= n_rows) return;
      if (kFromPairs) {
        __align__(16) __nv_bfloat16 fb[kIn / 2];
        const int sidx = a.ps[frow];
        const SrcPrep P = a.sprep ? a.sprep[sidx - a.sprep_base] : source_prep(a.fg, a.src[sidx]);
        const float4 c = a.fg.dom[a.pd[frow]];
        if (cg == 0)
          pair_features_half<0>(a.fg, P, c, fb);
        else
          pair_features_half<1>(a.fg, P, c, fb);
#pragma unroll
        for (int i = 0; i < kFeatVecs; ++i) fv[i] = *reinterpret_cast<const uint4*>(fb + 8 * i);
      } else if (cg == 0) {
#pragma unroll
        for (int i = 0; i < kFeatVecs; ++i)
          fv[i] = *reinterpret_cast<const uint4*>(a.feat + frow * kIn + 8 * i);
        if (kTrain) {  // the features K-tiled, the first layer's weight-gradient operand
#pragma unroll
          for (int i = 0; i < kFeatVecs; ++i) {
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&fv[i]);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              *reinterpret_cast<__nv_bfloat16*>(
                  a.x_t + kt_off((uint32_t)(8 * i + j), (uint32_t)frow, kIn)) = e[j];
          }
        }
      }
    };
    auto store_features = [&]() {
      if (kFromPairs) {
#pragma unroll
        for (int i = 0; i < kFeatVecs; ++i)
          *reinterpret_cast<uint4*>(sH + tc::tile_off(r, cg * (kIn / 2) + 8 * i, kIn)) = fv[i];
      } else if (cg == 0) {
#pragma unroll
        for (int i = 0; i < kFeatVecs; ++i)
          *reinterpret_cast<uint4*>(sH + tc::tile_off(r, 8 * i, kIn)) = fv[i];
      }
    };
    if ((int64_t)blockIdx.x < n_tiles) {
      gather_features(blockIdx.x);
      store_features();
      tc::fence_smem_async();
      tc::fence_before_sync();
      tc::mbar_arrive(&in_ready[h]);
    }
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int64_t row = t * kRows + h * kHalf + r;
      const bool valid = row < n_rows;
      const bool has_next = t + gridDim.x < n_tiles;
      float zh = 0.0f;  // head: this column group's part of w5 . h4
      // one layer's epilogue; whether it is the last layer (the head, no
      // activations stored) is a compile-time argument, so the column loop
      // carries no branch on it (2 % of the kernel's time)
      auto run_layer = [&](int layer, auto last_tag) -> bool {
        // warp-uniform outcome: the TMEM loads below are warp-collective
        const bool got = tc::mbar_wait(&acc_full[h], acc_phase & 1, kWaitTries) &&
                         !*(volatile int*)&abort_flag;
        if (!__all_sync(0xffffffffu, got)) return false;
        ++acc_phase;
        __syncwarp();
        tc::fence_after_sync();
        constexpr bool last = decltype(last_tag)::value;
        // the last layer's MMAs have read the activations: the next tile's features
        if (last && has_next) store_features();
        // the same biases for the warp's 32 rows: a broadcast from the constant
        // cache (inference) or shared memory (training)
        const float* hbias = (kTrain ? par : hbias_par.v) + layer * kHid + c_begin;
        const float* w5 = par + L::kW5 + c_begin;
        // kEpiCols columns: bias, SiLU, BF16; into shared memory (or the head)
        auto consume = [&](const uint32_t (&raw)[kEpiCols], int c0) {
          uint32_t packed[kEpiCols / 2];
          uint32_t zpk[4];
#pragma unroll
          for (int j4 = 0; j4 < kEpiCols / 4; ++j4) {
            const float4 hb = *reinterpret_cast<const float4*>(hbias + c0 + 4 * j4);
            // z / 2 = acc / 2 + b / 2, two columns per instruction
            const float2 h01 = ffma2(make_float2(__uint_as_float(raw[4 * j4 + 0]),
                                                 __uint_as_float(raw[4 * j4 + 1])),
                                     make_float2(0.5f, 0.5f), make_float2(hb.x, hb.y));
            const float2 h23 = ffma2(make_float2(__uint_as_float(raw[4 * j4 + 2]),
                                                 __uint_as_float(raw[4 * j4 + 3])),
                                     make_float2(0.5f, 0.5f), make_float2(hb.z, hb.w));
            const float hz[4] = {h01.x, h01.y, h23.x, h23.y};
            float y[4];
            if (kMode == kModeSiluFast) {
              // silu(2h) = h (1 + tanh h) = h tanh h + h, two columns per FMA
              const float2 y01 = ffma2(h01, make_float2(tanh_approx(h01.x), tanh_approx(h01.y)), h01);
              const float2 y23 = ffma2(h23, make_float2(tanh_approx(h23.x), tanh_approx(h23.y)), h23);
              y[0] = y01.x;
              y[1] = y01.y;
              y[2] = y23.x;
              y[3] = y23.y;
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (kMode == kModeHardSwish)  // z t with t = sat(z / 6 + 1/2) = sat(h / 3 + 1/2)
                  y[i] = (hz[i] + hz[i]) * __saturatef(fmaf(hz[i], 1.0f / 3.0f, 0.5f));
                else
                  y[i] = silu_exact(hz[i] + hz[i]);
            }
            packed[2 * j4] = pack_bf16(y[0], y[1]);
            packed[2 * j4 + 1] = pack_bf16(y[2], y[3]);
            if (kTrain) {
              zpk[2 * (j4 & 1)] = pack_bf16(hz[0] + hz[0], hz[1] + hz[1]);
              zpk[2 * (j4 & 1) + 1] = pack_bf16(hz[2] + hz[2], hz[3] + hz[3]);
              if ((j4 & 1) && valid) {
                const size_t o = (size_t)row * kHid + c_begin + c0 + 4 * (j4 - 1);
                *reinterpret_cast<uint4*>(a.z_out[layer] + o) =
                    make_uint4(zpk[0], zpk[1], zpk[2], zpk[3]);
                if (last)
                  *reinterpret_cast<uint4*>(a.h_out[layer] + o) = make_uint4(
                      packed[2 * j4 - 2], packed[2 * j4 - 1], packed[2 * j4], packed[2 * j4 + 1]);
              }
            }
          }
          if (kTrain && !last && valid) {
            // activations K-tiled ([256][n]): a warp's 32 rows of one column
            // land in four 16-byte runs
            unsigned char* ht = reinterpret_cast<unsigned char*>(a.h_out[layer]);
#pragma unroll
            for (int j = 0; j < kEpiCols / 2; ++j) {
              const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&packed[j]);
              const uint32_t m = (uint32_t)(c_begin + c0 + 2 * j);
              *reinterpret_cast<__nv_bfloat16*>(ht + kt_off(m, (uint32_t)row, kHid)) = __low2bfloat16(v);
              *reinterpret_cast<__nv_bfloat16*>(ht + kt_off(m + 1, (uint32_t)row, kHid)) =
                  __high2bfloat16(v);
            }
          }
          if (!last) {
#pragma unroll
            for (int i = 0; i < kEpiCols / 8; ++i)
              *reinterpret_cast<uint4*>(sH + tc::tile_off(r, c_begin + c0 + 8 * i, kHid)) =
                  make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2],
                             packed[4 * i + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < kEpiCols / 2; ++j) {
              const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&packed[j]);
              zh = fmaf(__low2float(v), w5[c0 + 2 * j], zh);
              zh = fmaf(__high2float(v), w5[c0 + 2 * j + 1], zh);
            }
          }
        };
        // two register sets: the next TMEM load is in flight while one is converted
        uint32_t ra[kEpiCols], rb[kEpiCols];
        epi_ld(tacc + 0, ra);
        tc::tmem_wait_ld(ra);
#pragma unroll
        for (int c0 = 0; c0 < kColsPerWarp; c0 += 2 * kEpiCols) {
          epi_ld(tacc + c0 + kEpiCols, rb);
          consume(ra, c0);
          tc::tmem_wait_ld(rb);
          if (c0 + 2 * kEpiCols < kColsPerWarp) epi_ld(tacc + c0 + 2 * kEpiCols, ra);
          consume(rb, c0 + kEpiCols);
          if (c0 + 2 * kEpiCols < kColsPerWarp) tc::tmem_wait_ld(ra);
        }
        if (!last || has_next) {
          // activations (or the next tile's features) written and the
          // accumulator read: the half's next MMA may start
          tc::fence_smem_async();
          tc::fence_before_sync();
          tc::mbar_arrive(&in_ready[h]);
        }
        return true;
      };
      bool lok = true;
      for (int layer = 0; layer < kLayers - 1 && lok; ++layer) lok = run_layer(layer, std::false_type{});
      if (lok && has_next) gather_features(t + gridDim.x);
      if (lok) lok = run_layer(kLayers - 1, std::true_type{});
      if (!lok) ok = false;
      if (!ok) break;
      // the head: column group 1 hands its partial sum to group 0
      if (cg == 1) {
        zpart[h * kHalf + r] = zh;
        tc::mbar_arrive(hb);
        continue;
      }
      const bool got = tc::mbar_wait(hb, head_phase & 1, kWaitTries);
      ++head_phase;
      if (!got) {
        ok = false;
        break;
      }
      zh += zpart[h * kHalf + r];
      if (valid) {
        const float z = zh + *a.b5;
        if (kFromPairs) {
          const int s = a.ps[row], d = a.pd[row];
          const float lam = a.nph[s] * softplus(z);
          if (a.dom_sum) atomicAdd(a.dom_sum + d, (double)lam);
          if (a.lambda_out) a.lambda_out[(size_t)s * a.n_dom + d] = lam;
        } else if (!kTrain) {
          a.lambda[row] = a.nph[row] * softplus(z);
        }
      }
    }
    if (!ok) {
      atomicExch(&abort_flag, 1);
      atomicOr(a.err, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}


// Backward pass of the hidden layers for training, fused like the forward:
// per 256-row tile, dL/dz of the last hidden layer (from the head) becomes
// the A operand; three MMA layers against the transposed weights W4^T, W3^T,
// W2^T give dL/dz of layers 3, 2, 1:
//   dz_{l-1} = bf16((dz_l . W_l) * silu'(z_{l-1}))
// each written back into shared memory (the next A operand) and, transposed
// ([256][n], the weight-gradient GEMM's operand), to global memory.  Same warp roles, ping-pong and bounded
// waits as k_mlp_fused; the weight image holds 4 chunks per transposed layer.
constexpr int kBwdLayers = kLayers - 1;
constexpr int kBwdChunksPerTile = 2 * kBwdLayers * kChunksPerLayer;

__global__ void __launch_bounds__(kThreads, 1) k_mlp_bwd(BwdArgs a) {
  constexpr int kStages = kBwdStages;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], in_ready[2], done;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = (a.n + kRows - 1) / kRows;
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int h = 0; h < 2; ++h) {
      tc::mbar_init(&acc_full[h], 1);
      tc::mbar_init(&in_ready[h], kEpiThreads / 2);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int jt = 0; jt < kBwdChunksPerTile; ++jt, ++it) {
          // job order (layer step j, half); step j's chunk c is 8 j + c
          const int j = jt / (2 * kChunksPerLayer), c = jt % kChunksPerLayer;
          const uint32_t s = it % kStages;
          if (it >= (uint32_t)kStages) {
            if (!tc::mbar_wait(&empty[s], ((it / kStages) - 1) & 1, kWaitTries) ||
                *(volatile int*)&abort_flag) {
              ok = false;
              break;
            }
          }
          tc::mbar_arrive_expect_tx(&full[s], kChunkBytes);
          tc::bulk_g2s(smem + kOffRing + s * kChunkBytes,
                       a.wpack + (size_t)(j * kChunksPerLayer + c) * kChunkBytes, kChunkBytes,
                       &full[s]);
        }
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        atomicOr(a.err, 1);
      }
      const uint32_t last = it < (uint32_t)kStages ? it : (uint32_t)kStages;
      for (uint32_t q = 0; q < last; ++q) {
        const uint32_t i = it - 1 - q;
        tc::mbar_wait(&full[i % kStages], (i / kStages) & 1, kWaitTries);
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kHalf, kHid);
      const uint32_t sh = tc::smem_u32(smem + kOffH);
      const uint32_t ring = tc::smem_u32(smem + kOffRing);
      uint32_t it = 0, in_phase[2] = {0u, 0u};
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int job = 0; job < 2 * kBwdLayers && ok; ++job) {
          const int h = job & 1;
          if (!tc::mbar_wait(&in_ready[h], in_phase[h] & 1, kWaitTries) ||
              *(volatile int*)&abort_flag) {
            ok = false;
            break;
          }
          ++in_phase[h];
          tc::fence_after_sync();
          for (int c = 0; c < kChunksPerLayer; ++c, ++it) {
            const uint32_t s = it % kStages;
            if (!tc::mbar_wait(&full[s], (it / kStages) & 1, kWaitTries)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t b0 = ring + s * kChunkBytes;
#pragma unroll
            for (int kk = 0; kk < kChunkK / 16; ++kk) {
              const uint32_t k0 = c * kChunkK + kk * 16;
              tc::mma_bf16(tmem + h * kHid,
                           tc::smem_desc(sh + h * kHalfBytes + k0 * 16, 128, kHid * 16),
                           tc::smem_desc(b0 + kk * 256, 128, kChunkK * 16), idesc,
                           (c > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[s]);
          }
          tc::mma_commit(&acc_full[h]);
        }
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        atomicOr(a.err, 1);
      }
      tc::mma_commit(&done);
      tc::mbar_wait(&done, 0, kWaitTries);
    }
  } else {
    const int q = warp & 3, h = (warp >> 2) & 1, cg = warp >> 3;
    const int r = q * 32 + lane;
    const int c_begin = cg * kColsPerWarp;
    unsigned char* sH = smem + kOffH + h * kHalfBytes;
    const uint32_t tacc =
        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * kHid) + (uint32_t)c_begin;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int64_t row = t * kRows + h * kHalf + r;
      const bool valid = row < a.n;
      // dL/dz of the last hidden layer: this warp's 128 columns of the row
      {
        const __nv_bfloat16* src = a.dz[kBwdLayers] + (size_t)row * kHid + c_begin;
#pragma unroll 4
        for (int i = 0; i < kColsPerWarp / 8; ++i) {
          const uint4 v = valid ? *reinterpret_cast<const uint4*>(src + 8 * i)
                                : make_uint4(0, 0, 0, 0);
          *reinterpret_cast<uint4*>(sH + tc::tile_off(r, c_begin + 8 * i, kHid)) = v;
          if (valid) {  // and K-tiled, the last layer's weight-gradient operand
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              *reinterpret_cast<__nv_bfloat16*>(
                  a.dz3_t + kt_off((uint32_t)(c_begin + 8 * i + j), (uint32_t)row, kHid)) = e[j];
          }
        }
        tc::fence_smem_async();
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&in_ready[h]);
      for (int j = 0; j < kBwdLayers; ++j) {
        const int lo = kBwdLayers - 1 - j;  // layer whose dz this step produces
        const bool got = tc::mbar_wait(&acc_full[h], acc_phase & 1, kWaitTries) &&
                         !*(volatile int*)&abort_flag;
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        ++acc_phase;
        __syncwarp();
        tc::fence_after_sync();
        const __nv_bfloat16* zrow = a.z[lo] + (size_t)row * kHid + c_begin;
        __nv_bfloat16* dzt = a.dz[lo];
        const bool last = j == kBwdLayers - 1;
        auto consume = [&](const uint32_t (&raw)[kEpiCols], int c0) {
          uint32_t packed[kEpiCols / 2];
#pragma unroll
          for (int i = 0; i < kEpiCols / 8; ++i) {
            uint4 zv = make_uint4(0, 0, 0, 0);
            if (valid) zv = *reinterpret_cast<const uint4*>(zrow + c0 + 8 * i);
            const uint32_t zw[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const __nv_bfloat162 z2 = *reinterpret_cast<const __nv_bfloat162*>(&zw[k]);
              const int e = 8 * i + 2 * k;
              packed[4 * i + k] =
                  pack_bf16(__uint_as_float(raw[e]) * act_grad(a.act, __low2float(z2)),
                            __uint_as_float(raw[e + 1]) * act_grad(a.act, __high2float(z2)));
            }
          }
          if (!last) {
#pragma unroll
            for (int i = 0; i < kEpiCols / 8; ++i)
              *reinterpret_cast<uint4*>(sH + tc::tile_off(r, c_begin + c0 + 8 * i, kHid)) =
                  make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2],
                             packed[4 * i + 3]);
          }
          if (valid) {
            // dL/dz K-tiled ([256][n]), the weight-gradient kernel's A operand
            unsigned char* dt = reinterpret_cast<unsigned char*>(dzt);
#pragma unroll
            for (int j = 0; j < kEpiCols / 2; ++j) {
              const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&packed[j]);
              const uint32_t m = (uint32_t)(c_begin + c0 + 2 * j);
              *reinterpret_cast<__nv_bfloat16*>(dt + kt_off(m, (uint32_t)row, kHid)) = __low2bfloat16(v);
              *reinterpret_cast<__nv_bfloat16*>(dt + kt_off(m + 1, (uint32_t)row, kHid)) =
                  __high2bfloat16(v);
            }
          }
        };
        // two register sets: the next TMEM load is in flight while one is converted
        uint32_t ra[kEpiCols], rb[kEpiCols];
        epi_ld(tacc + 0, ra);
        tc::tmem_wait_ld(ra);
#pragma unroll
        for (int c0 = 0; c0 < kColsPerWarp; c0 += 2 * kEpiCols) {
          epi_ld(tacc + c0 + kEpiCols, rb);
          consume(ra, c0);
          tc::tmem_wait_ld(rb);
          if (c0 + 2 * kEpiCols < kColsPerWarp) epi_ld(tacc + c0 + 2 * kEpiCols, ra);
          consume(rb, c0 + kEpiCols);
          if (c0 + 2 * kEpiCols < kColsPerWarp) tc::tmem_wait_ld(ra);
        }
        if (!last) {
          tc::fence_smem_async();
          tc::fence_before_sync();
          tc::mbar_arrive(&in_ready[h]);
        }
      }
    }
    if (!ok) {
      atomicExch(&abort_flag, 1);
      atomicOr(a.err, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// The transposed hidden weights in the ring's chunk layout, for the backward
// pass: step j uses W_l^T with l = 3 - j (0-based layers), chunk c holding
// the outputs 64c .. 64c + 63 of W_l as K: element (in n, out k) of W_l^T at
// tile_off(n, k - 64c, 64) of its 32 KB block.
__global__ void k_pack_bwd(const __nv_bfloat16* w2, const __nv_bfloat16* w3,
                           const __nv_bfloat16* w4, unsigned char* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one element
  if (i >= kBwdLayers * kHid * kHid) return;
  const int j = i / (kHid * kHid);
  const int rem = i % (kHid * kHid);
  const int k = rem / kHid, n = rem % kHid;  // W_l[k][n]: output k, input n
  const __nv_bfloat16* w = j == 0 ? w4 : (j == 1 ? w3 : w2);
  const int c = k / kChunkK;
  unsigned char* dst = out + (size_t)(j * kChunksPerLayer + c) * kChunkBytes +
                       tc::tile_off(n, k - c * kChunkK, kChunkK);
  *reinterpret_cast<__nv_bfloat16*>(dst) = w[rem];
}

// Weight gradients of one layer: dw[256][nb] += sum over the batch of
// dz^T . x, both operands K-tiled (one 64-row block of each is one bulk copy).
// Persistent CTAs take blocks round-robin; the two 128-row halves of dw
// accumulate in TMEM (2 nb columns) over the CTA's blocks, and each CTA
// stores its partial sums (zeros when it had no block) to partial[CTA][256][nb];
// k_reduce_dw adds them to dw.  Warps 0-3: TMEM
// readout; warp 4: producer (3-stage ring); warp 5: MMA issue.  Bounded waits.
constexpr int kDwStages = 3;
constexpr int kDwThreads = 192;
constexpr uint32_t kDwABytes = kHid * kKTile * 2;  // 32 KB
constexpr uint32_t kDwStageBytes = 2 * kDwABytes;  // A and B (B <= 32 KB)

__global__ void __launch_bounds__(kDwThreads, 1) k_dw(DwArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kDwStages], empty[kDwStages], acc_done;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_blocks = a.n / kKTile;
  const uint32_t b_bytes = (uint32_t)a.nb * kKTile * 2;
  const uint32_t ncols = a.nb == kHid ? 512u : 64u;  // 2 nb, a power of two >= 32
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDwStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&acc_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const int64_t mine = blockIdx.x < n_blocks ? (n_blocks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (warp == 4) {
    if (lane == 0) {
      uint32_t it = 0;
      for (int64_t q = blockIdx.x; q < n_blocks; q += gridDim.x, ++it) {
        const uint32_t s = it % kDwStages;
        if (it >= (uint32_t)kDwStages &&
            (!tc::mbar_wait(&empty[s], ((it / kDwStages) - 1) & 1, kWaitTries) ||
             *(volatile int*)&abort_flag)) {
          atomicExch(&abort_flag, 1);
          atomicOr(a.err, 1);
          break;
        }
        unsigned char* st = smem + s * kDwStageBytes;
        tc::mbar_arrive_expect_tx(&full[s], kDwABytes + b_bytes);
        tc::bulk_g2s(st, a.a + (size_t)q * kDwABytes, kDwABytes, &full[s]);
        tc::bulk_g2s(st + kDwABytes, a.b + (size_t)q * b_bytes, b_bytes, &full[s]);
      }
      const uint32_t last = it < (uint32_t)kDwStages ? it : (uint32_t)kDwStages;
      for (uint32_t q = 0; q < last; ++q) {
        const uint32_t i = it - 1 - q;
        tc::mbar_wait(&full[i % kDwStages], (i / kDwStages) & 1, kWaitTries);
      }
    }
  } else if (warp == 5) {
    if (lane == 0 && mine > 0) {
      const uint32_t idesc = tc::idesc_bf16(kHalf, (uint32_t)a.nb);
      const uint32_t base = tc::smem_u32(smem);
      bool ok = true;
      uint32_t it = 0;
      for (int64_t q = blockIdx.x; q < n_blocks && ok; q += gridDim.x, ++it) {
        const uint32_t s = it % kDwStages;
        if (!tc::mbar_wait(&full[s], (it / kDwStages) & 1, kWaitTries) ||
            *(volatile int*)&abort_flag) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t sa = base + s * kDwStageBytes, sb = sa + kDwABytes;
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
          for (int kk = 0; kk < kKTile / 16; ++kk)
            tc::mma_bf16(tmem + mb * a.nb,
                         tc::smem_desc(sa + mb * (kHalf / 8) * (kKTile * 16) + kk * 256, 128,
                                       kKTile * 16),
                         tc::smem_desc(sb + kk * 256, 128, kKTile * 16), idesc,
                         (it > 0 || kk > 0) ? 1u : 0u);
        tc::mma_commit(&empty[s]);
      }
      if (!ok) {
        atomicExch(&abort_flag, 1);
        atomicOr(a.err, 1);
      }
      tc::mma_commit(&acc_done);
    }
  } else {
    // warps 0-3: TMEM lanes 32 w .. + 31 = rows of each half of dw
    float* part = a.partial + (size_t)blockIdx.x * kHid * a.nb;
    const bool got = mine == 0 ||
                     (tc::mbar_wait(&acc_done, 0, kWaitTries) && !*(volatile int*)&abort_flag);
    if (__all_sync(0xffffffffu, got)) {
      __syncwarp();
      tc::fence_after_sync();
      for (int mb = 0; mb < 2; ++mb) {
        const int m = mb * kHalf + warp * 32 + lane;
        for (int c0 = 0; c0 < a.nb; c0 += 32) {
          float v[32];
          if (mine > 0) {
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mb * a.nb + c0), v);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0.0f;
          }
          float4* dst = reinterpret_cast<float4*>(part + (size_t)m * a.nb + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
    } else if (lane == 0) {
      atomicOr(a.err, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// dw[i] += sum over the CTAs of partial[c][i]
__global__ void k_reduce_dw(const float* partial, int parts, int size, float* dw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= size) return;
  float acc = 0.0f;
  for (int c = 0; c < parts; ++c) acc += partial[(size_t)c * size + i];
  dw[i] += acc;
}

__global__ void __launch_bounds__(256) k_rowsum_kt(const unsigned char* in, int R, int64_t n,
                                                    float* out) {
  __shared__ float part[8];
  const uint32_t r = blockIdx.x;
  float acc = 0.0f;
  for (int64_t g = threadIdx.x; g < n / 8; g += blockDim.x) {  // 8 consecutive batch rows
    const uint4 v = *reinterpret_cast<const uint4*>(in + kt_off(r, (uint32_t)(g * 8), (uint32_t)R));
    const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += __bfloat162float(e[j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += part[w];
    out[r] += t;
  }
}

// The weights in the ring's chunk layout: W1 ([256][32], one K-major 16 KB
// block), then each hidden layer (BF16 [256 out][256 in]) as 4 chunks of 64
// inputs, each one K-major 32 KB block; every chunk is staged by one bulk copy.
__global__ void k_pack_weights(const __nv_bfloat16* w1, const __nv_bfloat16* w2,
                               const __nv_bfloat16* w3, const __nv_bfloat16* w4,
                               unsigned char* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one 8-element group
  constexpr int kG1 = kHid * kIn / 8, kGh = kHid * kHid / 8;
  if (i >= kG1 + kHiddenGemms * kGh) return;
  if (i < kG1) {
    const int n = i / (kIn / 8), k = (i % (kIn / 8)) * 8;
    *reinterpret_cast<uint4*>(out + tc::tile_off(n, k, kIn)) =
        *reinterpret_cast<const uint4*>(w1 + n * kIn + k);
    return;
  }
  const int l = (i - kG1) / kGh;
  const int rem = (i - kG1) % kGh;
  const int n = rem / (kHid / 8), k = (rem % (kHid / 8)) * 8;
  const __nv_bfloat16* w = l == 0 ? w2 : (l == 1 ? w3 : w4);
  const int c = k / kChunkK;
  unsigned char* dst = out + (size_t)kW1Bytes + (size_t)(l * kChunksPerLayer + c) * kChunkBytes +
                       tc::tile_off(n, k - c * kChunkK, kChunkK);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(w + n * kHid + k);
}

}  // namespace

size_t packed_weight_bytes() {
  return (size_t)kW1Bytes + (size_t)kHiddenGemms * kChunksPerLayer * kChunkBytes;
}

cudaError_t launch_pack_weights(const __nv_bfloat16* const* w, unsigned char* out,
                                cudaStream_t st) {
  const int groups = kHid * kIn / 8 + kHiddenGemms * kHid * kHid / 8;
  k_pack_weights<<<(groups + 255) / 256, 256, 0, st>>>(w[0], w[1], w[2], w[3], out);
  return cudaGetLastError();
}

template <bool P, int E, bool T = false>
cudaError_t launch_variant(const FusedArgs& a, const HalfBias& hb, int g, cudaStream_t st) {
  constexpr uint32_t bytes = FwdLayout<T>::kSmemBytes;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_fused<P, E, T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_mlp_fused<P, E, T><<<g, kThreads, bytes, st>>>(a, hb);
  return cudaGetLastError();
}

size_t packed_bwd_bytes() { return (size_t)kBwdLayers * kChunksPerLayer * kChunkBytes; }

cudaError_t launch_pack_bwd(const __nv_bfloat16* const* w, unsigned char* out, cudaStream_t st) {
  const int n = kBwdLayers * kHid * kHid;
  k_pack_bwd<<<(n + 255) / 256, 256, 0, st>>>(w[1], w[2], w[3], out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_bwd(const BwdArgs& a, int grid, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const int64_t tiles = (a.n + kRows - 1) / kRows;
  const int g = (int)(tiles < grid ? tiles : grid);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBwdSmemBytes);
  if (e != cudaSuccess) return e;
  k_mlp_bwd<<<g, kThreads, kBwdSmemBytes, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dw(const DwArgs& a, int grid, cudaStream_t st) {
  const int64_t blocks = a.n / kKTile;
  if (blocks <= 0) return cudaSuccess;
  if (grid > a.partial_cap) grid = a.partial_cap;
  if (grid < 1 || (a.nb != kHid && a.nb != kIn) || a.n % kKTile) return cudaErrorInvalidValue;
  const int g = (int)(blocks < grid ? blocks : grid);
  const size_t smem = (size_t)kDwStages * kDwStageBytes;
  cudaError_t e = cudaFuncSetAttribute(k_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dw<<<g, kDwThreads, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int size = kHid * a.nb;
  k_reduce_dw<<<(size + 255) / 256, 256, 0, st>>>(a.partial, g, size, a.dw);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_kt(const unsigned char* in, int R, int64_t n, float* out,
                             cudaStream_t st) {
  if (R <= 0 || n <= 0) return cudaSuccess;
  k_rowsum_kt<<<R, 256, 0, st>>>(in, R, n, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_fused(const FusedArgs& a, const HalfBias* hb, bool from_pairs, int grid,
                             cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const int64_t tiles = (a.n + kRows - 1) / kRows;
  const int g = (int)(tiles < grid ? tiles : grid);
  const bool hs = a.act == kActHardSwish;
  static const HalfBias unused{};  // the training forward reads a.bias
  if (a.z_out[0])  // training forward: the activation evaluated exactly
    return hs ? launch_variant<false, kModeHardSwish, true>(a, unused, g, st)
              : launch_variant<false, kModeSiluExact, true>(a, unused, g, st);
  if (!hb) return cudaErrorInvalidValue;
  const int mode = hs ? kModeHardSwish : (a.exact_silu ? kModeSiluExact : kModeSiluFast);
  if (from_pairs)
    return mode == kModeHardSwish   ? launch_variant<true, kModeHardSwish>(a, *hb, g, st)
           : mode == kModeSiluExact ? launch_variant<true, kModeSiluExact>(a, *hb, g, st)
                                    : launch_variant<true, kModeSiluFast>(a, *hb, g, st);
  return mode == kModeHardSwish   ? launch_variant<false, kModeHardSwish>(a, *hb, g, st)
         : mode == kModeSiluExact ? launch_variant<false, kModeSiluExact>(a, *hb, g, st)
                                  : launch_variant<false, kModeSiluFast>(a, *hb, g, st);
}

}  // namespace mlp
