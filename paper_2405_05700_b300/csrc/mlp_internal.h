// Internal interface of the surrogate MLP kernels (mlp_fused.cu,
// mlp_kernels.cu) and its C ABI (pp_mlp.cu).  Not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pp.h"

namespace mlp {

// Plain tensor-core GEMM C = A . B^T (FP32), the debug entry point's kernel.
struct GemmArgs {
  const __nv_bfloat16* A;  // [M][lda], K contiguous
  const __nv_bfloat16* B;  // [N][ldb], K contiguous
  int M, N, K, lda, ldb, ldc;
  int bn;                  // N tile: multiple of 16, <= 256
  float* Cf;
  int* err;
};

size_t gemm_smem_bytes(int bn);
cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t st);

constexpr int kIn = 32;      // input features (10 named + 22 derived), the first MMA's K
constexpr int kHid = 256;    // hidden width
constexpr int kLayers = 4;   // hidden layers (Linear + SiLU)

// Geometry and ice the feature kernels read (device pointers).
struct FeatGeom {
  const float4* dom;         // [n_dom] (x, y, z, 0)
  const float4* layer;       // [L] (b, a, 1/b, 1/a), b geometric
  const float2* cum;         // [L] sums of (b_e, a) over the layers before each
  int n_dom, L;
  float z_top, dz, be_over_b;  // effective b_e = b * be_over_b
  float theta_c;             // Cherenkov angle (rad)
};

// fg.cum from fg.layer (one thread; L is small).
cudaError_t launch_ice_cum(const FeatGeom& fg, float2* cum, cudaStream_t st);

// Hidden-layer activations (the network's definition; the oracle states the same):
//   kActSilu       silu(z) = z / (1 + exp(-z))
//   kActHardSwish  hswish(z) = z * clamp(z / 6 + 1/2, 0, 1): no special-function
//                  operation, the derivative t + z / 6 inside (-3, 3), t outside
//                  (t = clamp(z / 6 + 1/2, 0, 1); at z = -3 and 3 the outer value)
constexpr int kActSilu = 0;
constexpr int kActHardSwish = 1;

__device__ __forceinline__ float act_grad(int act, float z) {
  if (act == kActHardSwish) {
    const float u = fmaf(z, 1.0f / 6.0f, 0.5f);
    const float t = __saturatef(u);
    return (u > 0.0f && u < 1.0f) ? fmaf(z, 1.0f / 6.0f, t) : t;
  }
  const float sg = 1.0f / (1.0f + __expf(-z));
  return sg * (1.0f + z * (1.0f - sg));
}

struct SrcPrep;  // per-source part of the features (mlp_features.cuh)

// The per-source part of the features of sources [s0, s0 + ns) into out[ns].
cudaError_t launch_src_prep(const FeatGeom& fg, const pp_source* src, int64_t s0, int64_t ns,
                            SrcPrep* out, cudaStream_t st);

// Features of pairs (source s, DOM d) as BF16 [n][32].
cudaError_t launch_features(const FeatGeom& fg, const pp_source* src, const int32_t* pair_src,
                            const int32_t* pair_dom, int64_t n, __nv_bfloat16* feat,
                            cudaStream_t st);

// Head with loss and gradients: Poisson NLL sum(lambda - n ln lambda) / n_total;
// dZ4 = dL/dz * w5 * silu'(z4) (BF16); dw5b5[0..255] += sum dL/dz * h,
// dw5b5[256] += sum dL/dz, loss (double) += the batch's loss sum / n_total.
// Per-block partial sums go to part[ceil(n / 64)][257] and lpart[ceil(n / 64)]
// (part_rows rows available) and are added in block order: deterministic.
cudaError_t launch_head_backward(const __nv_bfloat16* h, const __nv_bfloat16* z4, const float* w5,
                                 const float* b5, const float* nph, const float* cnt, int64_t n,
                                 float inv_n, __nv_bfloat16* dz4, float* dw5b5, double* loss,
                                 float* part, double* lpart, int64_t part_rows, int act,
                                 cudaStream_t st);
constexpr int kHeadPartCols = 257;  // W5 and b5
constexpr int kHeadPartPairs = 64;  // pairs per partial-sum row

// out[i] = in[rows[i]] for features [.][32], photons and counts; a row outside
// [0, n_rows) sets kGatherBadRow in *err and reads row 0.
constexpr int kGatherBadRow = 4;
cudaError_t launch_gather_rows(const __nv_bfloat16* feat, const float* nph, const float* cnt,
                               int64_t n_rows, const int64_t* rows, int64_t n,
                               __nv_bfloat16* feat_out, float* nph_out, float* cnt_out, int* err,
                               cudaStream_t st);

// Pairs of sources [s0, s0+ns) x DOMs within r_max into (ps, pd) in any order;
// *count += all of them (only the first max_out are written).
cudaError_t launch_near_pairs(const FeatGeom& fg, const pp_source* src, int64_t s0, int64_t ns,
                              float r_max, int64_t max_out, int32_t* ps, int32_t* pd,
                              unsigned long long* count, cudaStream_t st);
// The same for sources [0, ns) in (source, DOM) order; *count = all of them.
// Scratch: bcount[nb], boff[nb] with nb = near_pairs_ordered_blocks(ns * n_dom).
int64_t near_pairs_ordered_blocks(int64_t n_candidates);
cudaError_t launch_near_pairs_ordered(const FeatGeom& fg, const pp_source* src, int64_t ns,
                                      float r_max, int64_t max_out, int32_t* ps, int32_t* pd,
                                      unsigned long long* count, uint32_t* bcount,
                                      unsigned long long* boff, cudaStream_t st);
// Fused inference (mlp_fused.cu): rows are either pairs (features computed
// in the kernel; lambda summed per DOM and/or stored as [source][DOM]) or
// precomputed BF16 feature rows (lambda per row).  All feature and pair
// pointers 16-byte aligned.
struct FusedArgs {
  FeatGeom fg;
  const pp_source* src;          // pairs mode
  const SrcPrep* sprep;          // pairs mode, optional: sprep[s - sprep_base] for source s
  int64_t sprep_base;
  const int32_t* ps;
  const int32_t* pd;
  // pairs mode, optional: the row count in device memory (used up to n)
  const unsigned long long* n_dev;
  const __nv_bfloat16* feat;     // rows mode: [n][kIn]
  int64_t n;
  const unsigned char* wpack;    // W1..W4 in the ring's chunk layout
  int act;                       // kActSilu or kActHardSwish
  int exact_silu;                // SiLU: 1: z / (1 + exp(-z)); 0: one tanh.approx
  const float* bias[kLayers];
  const float* w5;
  const float* b5;
  const float* nph;              // per source (pairs) or per row
  double* dom_sum;               // pairs mode, may be null
  float* lambda_out;             // pairs mode [n_src][n_dom], may be null
  int n_dom;
  float* lambda;                 // rows mode (inference)
  // training forward (rows mode, exact SiLU, no lambda): each layer's BF16
  // pre-activations [n][256] and activations (layers 0-2 K-tiled [256][n],
  // layer 3 [n][256]); null for inference
  __nv_bfloat16* z_out[kLayers];
  __nv_bfloat16* h_out[kLayers];
  unsigned char* x_t;            // training: the features K-tiled [32][n]
  int* err;
};

size_t packed_weight_bytes();
cudaError_t launch_pack_weights(const __nv_bfloat16* const* w, unsigned char* out,
                                cudaStream_t st);
// The hidden layers' biases halved (b / 2, layer-major [4][256]).  Inference
// passes them to the fused kernel as a launch parameter: its epilogue reads
// them from the constant cache, which leaves the shared memory they would
// take to a third stage of the weight ring.
struct HalfBias {
  float v[kLayers * kHid];
};

// grid: the CTA count cap (one CTA per SM runs at a time).  hb: the halved
// biases of a.bias, required for inference; the training forward (a.z_out
// set) reads a.bias itself and ignores hb.
cudaError_t launch_mlp_fused(const FusedArgs& a, const HalfBias* hb, bool from_pairs, int grid,
                             cudaStream_t st);

// Fused backward of the hidden layers (training): from dz[3] (dL/dz of the
// last hidden layer, BF16 [n][256]) and the forward's pre-activations z[0..2]
// ([n][256]), writes dz[2], dz[1], dz[0] K-tiled ([256][n]).  wpack: the
// transposed hidden weights packed by launch_pack_bwd.
struct BwdArgs {
  int64_t n;
  int act;                       // kActSilu or kActHardSwish
  const unsigned char* wpack;
  const __nv_bfloat16* z[kLayers];
  __nv_bfloat16* dz[kLayers];
  unsigned char* dz3_t;          // dz[3] K-tiled [256][n], written while it is staged
  int* err;
};
size_t packed_bwd_bytes();
// w: the 4 BF16 weight matrices (w[1..3] used)
cudaError_t launch_pack_bwd(const __nv_bfloat16* const* w, unsigned char* out, cudaStream_t st);
cudaError_t launch_mlp_bwd(const BwdArgs& a, int grid, cudaStream_t st);

// K-tiled layout of a training matrix X[R][n] (R = 256 units or the 32
// features; K = the n batch rows, a multiple of 64): blocks of 64 batch rows,
// each the K-major core-matrix image of an MMA operand tile (R x 64 BF16), so
// that one bulk copy stages it.  Byte offset of element (r, k):
constexpr int kKTile = 64;
__host__ __device__ constexpr size_t kt_off(uint32_t r, uint32_t k, uint32_t R) {
  return (size_t)(k / kKTile) * ((size_t)R * kKTile * 2) + (size_t)(r >> 3) * (kKTile * 16) +
         ((k % kKTile) >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// out[r] += sum over the n batch rows of a K-tiled [R][n] matrix (FP32)
cudaError_t launch_rowsum_kt(const unsigned char* in, int R, int64_t n, float* out,
                             cudaStream_t st);
// Weight gradient dw[256][nb] += A . B^T over the batch: A = dL/dz^T (R = 256),
// B = the layer's input^T (R = nb: 256 or 32), both K-tiled over n rows.
struct DwArgs {
  const unsigned char* a;
  const unsigned char* b;
  int64_t n;
  int nb;
  float* dw;
  float* partial;  // [partial_cap][256][nb] FP32 scratch
  int partial_cap;  // CTAs the scratch holds (the grid is capped to it)
  int* err;
};
cudaError_t launch_dw(const DwArgs& a, int grid, cudaStream_t st);

// Adam on n parameters; writes the BF16 copy of the weights it updates.
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, __nv_bfloat16* pb,
                        cudaStream_t st);
cudaError_t launch_to_bf16(const float* in, int64_t n, __nv_bfloat16* out, cudaStream_t st);

}  // namespace mlp
