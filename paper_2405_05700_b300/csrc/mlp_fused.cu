// Fused surrogate inference: features, the four hidden layers and the Poisson
// head of 256 pairs per tile in one persistent kernel, the activations never
// leaving the SM.
//
// Per CTA (one per SM): two row halves of 128 pairs, each an M = 128 tcgen05
// MMA with its FP32 accumulator (256 columns) in TMEM, so one weight chunk
// feeds both halves.  The layer's input (features, then BF16 activations)
// sits in shared memory as the MMA's A operand; the hidden layers' weights
// stream from global memory (L2-resident, shared by every CTA) through a ring
// of 16 KB chunks filled by bulk copies.
//
//   warps 0-7 : epilogue (warp w: half w / 4, TMEM lanes 32 (w % 4) ..): features,
//               bias + SiLU to BF16 back into shared memory, head
//   warp 8    : producer of the weight ring
//   warp 9    : MMA issue (one thread)
//
// Every wait is bounded; a wait that runs out raises the CTA's abort flag and
// the device error flag, and every role then leaves its loop.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_features.cuh"
#include "mlp_internal.h"
#include "tc_gemm.cuh"

namespace mlp {

namespace {

constexpr int kRows = 256;                 // pairs per tile
constexpr int kHalf = 128;                 // rows per MMA
constexpr int kChunkK = 32;                // K per weight chunk
constexpr int kChunksPerLayer = kHid / kChunkK;
constexpr int kChunkBytes = kHid * kChunkK * 2;
constexpr int kStages = 5;
constexpr int kHiddenGemms = kLayers - 1;  // layers 2..4 stream their weights
constexpr int kChunksPerTile = kHiddenGemms * kChunksPerLayer;
constexpr int kEpiThreads = 256;
constexpr int kThreads = kEpiThreads + 64;
constexpr uint32_t kWaitTries = 1u << 22;

// dynamic shared memory
constexpr uint32_t kOffH = 0;                                  // 2 x [128][256] BF16 (features alias)
constexpr uint32_t kHalfBytes = kHalf * kHid * 2;
constexpr uint32_t kOffW1 = kOffH + 2 * kHalfBytes;             // [256][16] BF16
constexpr uint32_t kOffRing = kOffW1 + kHid * kIn * 2;
constexpr uint32_t kOffPar = kOffRing + kStages * kChunkBytes;  // biases [4][256], w5 [256] (FP32)
constexpr uint32_t kSmemBytes = kOffPar + (kLayers + 1) * kHid * 4;

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// silu(z) = z sigmoid(z) = z (1 + tanh(z / 2)) / 2: one SFU operation.
__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(h), h);
}

__device__ __forceinline__ float softplus(float z) { return z > 20.0f ? z : log1pf(__expf(z)); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <bool kFromPairs>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_fused(FusedArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full, in_ready, done;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = (a.n + kRows - 1) / kRows;

  // setup: TMEM (512 columns: both accumulators), barriers, resident parameters
  if (warp == 0) tc::tmem_alloc(&tslot, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&acc_full, 1);
    tc::mbar_init(&in_ready, kEpiThreads);
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    float* par = reinterpret_cast<float*>(smem + kOffPar);
    for (int i = threadIdx.x; i < kLayers * kHid; i += blockDim.x)
      par[i] = a.bias[i / kHid][i % kHid];
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) par[kLayers * kHid + i] = a.w5[i];
    // W1 as the first MMA's B operand: K-major, 16 columns
    for (int i = threadIdx.x; i < kHid * 2; i += blockDim.x) {
      const int n = i >> 1, k8 = (i & 1) * 8;
      *reinterpret_cast<uint4*>(smem + kOffW1 + tc::tile_off(n, k8, kIn)) =
          *reinterpret_cast<const uint4*>(a.w1 + n * kIn + k8);
    }
  }
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;

  if (warp == 8) {
    // ---------------------------------------------------------- producer --
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int j = 0; j < kChunksPerTile; ++j, ++it) {
          const uint32_t s = it % kStages;
          if (it >= (uint32_t)kStages) {
            if (!tc::mbar_wait(&empty[s], ((it / kStages) - 1) & 1, kWaitTries) ||
                *(volatile int*)&abort_flag) {
              ok = false;
              break;
            }
          }
          tc::mbar_arrive_expect_tx(&full[s], kChunkBytes);
          tc::bulk_g2s(smem + kOffRing + s * kChunkBytes, a.wpack + (size_t)j * kChunkBytes,
                       kChunkBytes, &full[s]);
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
  } else if (warp == 9) {
    // --------------------------------------------------------------- MMA --
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kHalf, kHid);
      const uint32_t sh = tc::smem_u32(smem + kOffH);
      const uint32_t sw1 = tc::smem_u32(smem + kOffW1);
      const uint32_t ring = tc::smem_u32(smem + kOffRing);
      uint32_t it = 0, in_phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int layer = 0; layer < kLayers && ok; ++layer) {
          if (!tc::mbar_wait(&in_ready, in_phase & 1, kWaitTries) ||
              *(volatile int*)&abort_flag) {
            ok = false;
            break;
          }
          ++in_phase;
          tc::fence_after_sync();
          if (layer == 0) {
            for (int h = 0; h < 2; ++h)
              tc::mma_bf16(tmem + h * kHid, tc::smem_desc(sh + h * kHalfBytes, 128, kIn * 16),
                           tc::smem_desc(sw1, 128, kIn * 16), idesc, 0u);
          } else {
            for (int c = 0; c < kChunksPerLayer; ++c, ++it) {
              const uint32_t s = it % kStages;
              if (!tc::mbar_wait(&full[s], (it / kStages) & 1, kWaitTries)) {
                ok = false;
                break;
              }
              tc::fence_after_sync();
              const uint32_t b0 = ring + s * kChunkBytes;
#pragma unroll
              for (int h = 0; h < 2; ++h)
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
          }
          tc::mma_commit(&acc_full);
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
    const int h = warp >> 2, q = warp & 3;
    const int r = q * 32 + lane;  // row within the half = TMEM lane
    unsigned char* sH = smem + kOffH + h * kHalfBytes;
    const float* par = reinterpret_cast<const float*>(smem + kOffPar);
    const uint32_t tacc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * kHid);
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int64_t row = t * kRows + h * kHalf + r;
      const bool valid = row < a.n;
      // features of this row as the first MMA's A operand (aliasing the activations)
      {
        uint4 f0 = make_uint4(0, 0, 0, 0), f1 = f0;
        if (valid) {
          if (kFromPairs) {
            __align__(16) __nv_bfloat16 fb[kIn];
            pair_features(a.fg, a.src[a.ps[row]], a.fg.dom[a.pd[row]], fb);
            f0 = *reinterpret_cast<const uint4*>(fb);
            f1 = *reinterpret_cast<const uint4*>(fb + 8);
          } else {
            f0 = *reinterpret_cast<const uint4*>(a.feat + row * kIn);
            f1 = *reinterpret_cast<const uint4*>(a.feat + row * kIn + 8);
          }
        }
        *reinterpret_cast<uint4*>(sH + tc::tile_off(r, 0, kIn)) = f0;
        *reinterpret_cast<uint4*>(sH + tc::tile_off(r, 8, kIn)) = f1;
      }
      tc::fence_smem_async();
      tc::fence_before_sync();
      tc::mbar_arrive(&in_ready);
      float zh = 0.0f;  // head: w5 . h4
      for (int layer = 0; layer < kLayers; ++layer) {
        // warp-uniform outcome: the TMEM loads below are warp-collective
        const bool got = tc::mbar_wait(&acc_full, acc_phase & 1, kWaitTries) &&
                         !*(volatile int*)&abort_flag;
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        ++acc_phase;
        __syncwarp();
        tc::fence_after_sync();
        const float* bias = par + layer * kHid;
        const float* w5 = par + kLayers * kHid;
        for (int c0 = 0; c0 < kHid; c0 += 32) {
          uint32_t raw[32];
          tc::tmem_ld32_nowait(tacc + c0, raw);
          tc::tmem_wait_ld();
          uint32_t packed[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float y0 = silu_fast(__uint_as_float(raw[2 * j]) + bias[c0 + 2 * j]);
            const float y1 = silu_fast(__uint_as_float(raw[2 * j + 1]) + bias[c0 + 2 * j + 1]);
            packed[j] = pack_bf16(y0, y1);
          }
          if (layer < kLayers - 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              *reinterpret_cast<uint4*>(sH + tc::tile_off(r, c0 + 8 * i, kHid)) =
                  make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2],
                             packed[4 * i + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&packed[j]);
              zh = fmaf(__low2float(v), w5[c0 + 2 * j], zh);
              zh = fmaf(__high2float(v), w5[c0 + 2 * j + 1], zh);
            }
          }
        }
        if (layer < kLayers - 1) {
          // activations written and accumulator read: the next layer may start
          tc::fence_smem_async();
          tc::fence_before_sync();
          tc::mbar_arrive(&in_ready);
        }
      }
      if (!ok) break;
      if (valid) {
        const float z = zh + *a.b5;
        if (kFromPairs) {
          const int s = a.ps[row], d = a.pd[row];
          const float lam = a.nph[s] * softplus(z);
          if (a.dom_sum) atomicAdd(a.dom_sum + d, (double)lam);
          if (a.lambda_out) a.lambda_out[(size_t)s * a.n_dom + d] = lam;
        } else {
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

// Hidden-layer weights (BF16 [256 out][256 in] each) into the ring's chunk
// layout: layer l, chunk c (inputs 32c .. 32c + 31) is one K-major 16 KB
// block, so that one bulk copy stages it.
__global__ void k_pack_hidden(const __nv_bfloat16* w2, const __nv_bfloat16* w3,
                              const __nv_bfloat16* w4, unsigned char* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one 8-element group
  if (i >= kHiddenGemms * kHid * kHid / 8) return;
  const int l = i / (kHid * kHid / 8);
  const int rem = i % (kHid * kHid / 8);
  const int n = rem / (kHid / 8), k = (rem % (kHid / 8)) * 8;
  const __nv_bfloat16* w = l == 0 ? w2 : (l == 1 ? w3 : w4);
  const int c = k / kChunkK;
  unsigned char* dst = out + (size_t)(l * kChunksPerLayer + c) * kChunkBytes +
                       tc::tile_off(n, k - c * kChunkK, kChunkK);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(w + n * kHid + k);
}

}  // namespace

size_t packed_hidden_bytes() { return (size_t)kHiddenGemms * kChunksPerLayer * kChunkBytes; }

cudaError_t launch_pack_hidden(const __nv_bfloat16* w2, const __nv_bfloat16* w3,
                               const __nv_bfloat16* w4, unsigned char* out, cudaStream_t st) {
  const int groups = kHiddenGemms * kHid * kHid / 8;
  k_pack_hidden<<<(groups + 255) / 256, 256, 0, st>>>(w2, w3, w4, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_fused(const FusedArgs& a, bool from_pairs, int grid, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  const int64_t tiles = (a.n + kRows - 1) / kRows;
  const int g = (int)(tiles < grid ? tiles : grid);
  cudaError_t e;
  if (from_pairs) {
    e = cudaFuncSetAttribute(k_mlp_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e == cudaSuccess) k_mlp_fused<true><<<g, kThreads, kSmemBytes, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_mlp_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e == cudaSuccess) k_mlp_fused<false><<<g, kThreads, kSmemBytes, st>>>(a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mlp
