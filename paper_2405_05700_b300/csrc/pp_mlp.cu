// The learned surrogate behind the C ABI: an MLP from (source, DOM) pair
// features to the expected number of photons the DOM receives, trained on the
// propagator's own hit counts.  BF16 weights and activations, FP32
// accumulation on the tensor cores (the fused tcgen05 kernels of mlp_fused.cu
// for inference and the training forward / backward, the GEMM of
// mlp_kernels.cu for the weight gradients), FP32 master weights and Adam state.
//
//   h1 = silu(W1 x + b1), h2..h4 = silu(Wi h + bi), z = w5 . h4 + b5,
//   lambda = n_photons * softplus(z),  loss = mean(lambda - n ln lambda)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "mlp_features.cuh"
#include "mlp_internal.h"
#include "pp_nvtx.h"
#include "pp.h"
#include "pp_internal.h"

using namespace mlp;

namespace {

// Flat parameter layout (FP32): W1 [256][32], b1, W2 [256][256], b2, W3, b3,
// W4, b4, w5 [256], b5.
constexpr int64_t kOffW1 = 0;
constexpr int64_t kOffB1 = kOffW1 + kHid * kIn;
constexpr int64_t kOffW2 = kOffB1 + kHid;
constexpr int64_t kHidBlock = (int64_t)kHid * kHid + kHid;  // one hidden layer's W and b
constexpr int64_t kOffW5 = kOffW2 + 3 * kHidBlock;
constexpr int64_t kOffB5 = kOffW5 + kHid;
constexpr int64_t kNParams = kOffB5 + 1;
static_assert(kNParams == PP_MLP_N_PARAMS, "parameter count");

int64_t off_w(int layer) { return layer == 0 ? kOffW1 : kOffW2 + (layer - 1) * kHidBlock; }
int64_t off_b(int layer) { return layer == 0 ? kOffB1 : off_w(layer) + (int64_t)kHid * kHid; }

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}

}  // namespace

struct pp_mlp {
  pp_ctx* ctx = nullptr;
  ppk::LaunchView view{};
  FeatGeom fg{};
  int max_batch = 0;
  int64_t max_rows = 0;
  std::string last_error = "no error";
  // parameters
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* wb[kLayers] = {};   // BF16 weights of the 4 GEMM layers
  int64_t step = 0;
  // training activations [max_batch][256]
  __nv_bfloat16* z[kLayers] = {};
  __nv_bfloat16* h[kLayers] = {};
  __nv_bfloat16* dz[kLayers] = {};  // dL/dz of each layer (pre-activation) [max_batch][256]
  __nv_bfloat16 *t1 = nullptr, *t2 = nullptr;
  double* loss = nullptr;
  int* err = nullptr;
  // inference: hidden weights in the fused kernel's chunk layout (repacked
  // when the weights change), the pair list [max_rows]
  unsigned char* wpack = nullptr;
  int64_t weights_version = 0, packed_version = -1;
  // inference: the hidden biases / 2, the fused kernel's launch parameter
  // (read back from the FP32 masters when the weights change)
  HalfBias hbias{};
  int64_t hbias_version = -1;
  unsigned char* wpack_bwd = nullptr;  // transposed hidden weights for the backward kernel
  float* dw_part = nullptr;            // per-CTA weight-gradient partial sums
  __nv_bfloat16* bfeat = nullptr;      // batch gathered from chosen training rows [max_batch][32]
  float *bnph = nullptr, *bcnt = nullptr;
  float* head_part = nullptr;          // head backward: per-block partial sums of dW5, db5
  double* head_lpart = nullptr;        // and of the loss
  int64_t packed_bwd_version = -1;
  int exact_silu = 0;
  int act = kActSilu;
  float2* ice_cum = nullptr;
  int sms = 0;
  int32_t *ps = nullptr, *pd = nullptr;
  unsigned long long* count = nullptr;
  SrcPrep* sprep = nullptr;            // per-source feature part of one dom_sums pass
  int64_t sprep_cap = 0;
  // ordered pair search: per-block counts and offsets (grown on demand)
  // dom_sums: each pass's pair count (grown on demand)
  unsigned long long* pass_count = nullptr;
  int64_t pass_cap = 0;
  uint32_t* near_bcount = nullptr;
  unsigned long long* near_boff = nullptr;
  int64_t near_cap = 0;
};

namespace {

int mfail(pp_mlp* m, int code, const std::string& msg) {
  m->last_error = msg;
  return code;
}

#define PP_MLP_CUDA(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) return mfail(m, PP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// BF16 copies of the weights from the FP32 masters.
int refresh_bf16(pp_mlp* m, cudaStream_t st) {
  PP_MLP_CUDA(launch_to_bf16(m->p + kOffW1, (int64_t)kHid * kIn, m->wb[0], st));
  for (int l = 1; l < kLayers; ++l)
    PP_MLP_CUDA(launch_to_bf16(m->p + off_w(l), (int64_t)kHid * kHid, m->wb[l], st));
  return PP_OK;
}

int ensure_packed(pp_mlp* m, cudaStream_t st) {
  if (m->packed_version == m->weights_version) return PP_OK;
  PP_MLP_CUDA(launch_pack_weights(m->wb, m->wpack, st));
  m->packed_version = m->weights_version;
  return PP_OK;
}

// The halved biases for an inference launch.  After the weights change (set,
// restored or trained) they are read back once, so that call waits for the
// stream's earlier work.
int ensure_hbias(pp_mlp* m, cudaStream_t st) {
  if (m->hbias_version == m->weights_version) return PP_OK;
  HalfBias raw;
  for (int l = 0; l < kLayers; ++l)
    PP_MLP_CUDA(cudaMemcpyAsync(raw.v + l * kHid, m->p + off_b(l), sizeof(float) * kHid,
                                cudaMemcpyDeviceToHost, st));
  PP_MLP_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < kLayers * kHid; ++i) m->hbias.v[i] = 0.5f * raw.v[i];
  m->hbias_version = m->weights_version;
  return PP_OK;
}

FusedArgs fused_args(pp_mlp* m) {
  FusedArgs a{};
  a.fg = m->fg;
  a.wpack = m->wpack;
  a.exact_silu = m->exact_silu;
  a.act = m->act;
  for (int l = 0; l < kLayers; ++l) a.bias[l] = m->p + off_b(l);
  a.w5 = m->p + kOffW5;
  a.b5 = m->p + kOffB5;
  a.n_dom = m->fg.n_dom;
  a.err = m->err;
  return a;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Training forward through the fused kernel: every layer's BF16
// pre-activations m->z and activations m->h (exact SiLU, as the gradients
// assume).
int forward_train(pp_mlp* m, const __nv_bfloat16* x0, int n, cudaStream_t st) {
  int rc;
  if ((rc = ensure_packed(m, st))) return rc;
  FusedArgs a = fused_args(m);
  a.feat = x0;
  a.n = n;
  a.exact_silu = 1;
  for (int l = 0; l < kLayers; ++l) {
    a.z_out[l] = m->z[l];
    a.h_out[l] = m->h[l];
  }
  a.x_t = reinterpret_cast<unsigned char*>(m->t2);
  PP_MLP_CUDA(launch_mlp_fused(a, nullptr, false, m->sms, st));
  return PP_OK;
}

// Forward + backward of one batch: gradients into m->g (zeroed), loss added.
int forward_backward(pp_mlp* m, const __nv_bfloat16* x0, const float* nph, const float* cnt,
                     int n, cudaStream_t st) {
  int rc;
  PP_MLP_CUDA(cudaMemsetAsync(m->g, 0, sizeof(float) * kNParams, st));
  if ((rc = forward_train(m, x0, n, st))) return rc;
  static_assert(kOffB5 == kOffW5 + kHid, "W5 and b5 are adjacent");
  PP_MLP_CUDA(launch_head_backward(m->h[3], m->z[3], m->p + kOffW5, m->p + kOffB5, nph, cnt, n,
                                   1.0f / (float)n, m->dz[3], m->g + kOffW5, m->loss, m->head_part,
                                   m->head_lpart, m->max_batch / kHeadPartPairs, m->act, st));
  // dz_{l-1} = (dz_l . W_l) * silu'(z_{l-1}) for l = 3, 2, 1: one fused kernel
  if (m->packed_bwd_version != m->weights_version) {
    PP_MLP_CUDA(launch_pack_bwd(m->wb, m->wpack_bwd, st));
    m->packed_bwd_version = m->weights_version;
  }
  BwdArgs b{};
  b.n = n;
  b.act = m->act;
  b.wpack = m->wpack_bwd;
  b.dz3_t = reinterpret_cast<unsigned char*>(m->t1);
  for (int l = 0; l < kLayers; ++l) {
    b.z[l] = m->z[l];
    b.dz[l] = m->dz[l];
  }
  b.err = m->err;
  PP_MLP_CUDA(launch_mlp_bwd(b, m->sms, st));
  // dW_l = dz_l^T . x_l and db_l = sum dz_l over the batch, from K-tiled
  // operands the fused kernels left: dz_0..3, the features and h_0..2
  auto* dz3t = reinterpret_cast<unsigned char*>(m->t1);
  auto* x0t = reinterpret_cast<unsigned char*>(m->t2);
  for (int l = kLayers - 1; l >= 0; --l) {
    DwArgs d{};
    d.a = l == kLayers - 1 ? dz3t : reinterpret_cast<const unsigned char*>(m->dz[l]);
    d.b = l == 0 ? x0t : reinterpret_cast<const unsigned char*>(m->h[l - 1]);
    d.n = n;
    d.nb = l == 0 ? kIn : kHid;
    d.dw = m->g + off_w(l);
    d.partial = m->dw_part;
    d.partial_cap = m->sms;
    d.err = m->err;
    PP_MLP_CUDA(launch_rowsum_kt(d.a, kHid, n, m->g + off_b(l), st));
    PP_MLP_CUDA(launch_dw(d, m->sms, st));
  }
  return PP_OK;
}

int check_batch(pp_mlp* m, int64_t n, const void* d_feat) {
  if (n < kKTile || n > m->max_batch || n % kKTile)
    return mfail(m, PP_EINVAL, "training batch must be a multiple of 64 in [64, max_batch]");
  if (!aligned16(d_feat)) return mfail(m, PP_EINVAL, "features must be 16-byte aligned");
  return PP_OK;
}

// One Adam step on a batch already in device memory (features 16-byte aligned).
int train_step(pp_mlp* m, const __nv_bfloat16* feat, const float* nph, const float* cnt,
               int64_t n, float lr, cudaStream_t st);

int mlp_sync(pp_mlp* m, cudaStream_t st) {
  PP_MLP_CUDA(cudaStreamSynchronize(st));
  int flag = 0;
  PP_MLP_CUDA(cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    PP_MLP_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    if (flag & kGatherBadRow)
      return mfail(m, PP_EDEVICE, "a training row index was outside the training set");
    return mfail(m, PP_EDEVICE, "a tensor-core wait ran out (device error flag)");
  }
  return PP_OK;
}

}  // namespace

extern "C" {

int pp_mlp_create(pp_ctx* ctx, int32_t max_batch, int64_t max_rows, pp_mlp** out) {
  if (!ctx || !out || max_batch < kKTile || max_batch % kKTile || max_rows < 1) return PP_EINVAL;
  *out = nullptr;
  pp_mlp* m = new pp_mlp();
  m->ctx = ctx;
  m->max_batch = max_batch;
  m->max_rows = max_rows;
  const int rc = ppk::with_launch_view(ctx, [&](const ppk::LaunchView& v) {
    m->view = v;
    ppk::attach_server(ctx, +1);  // keeps the context's tables in place
    return PP_OK;
  });
  if (rc) {
    delete m;
    return rc;
  }
  const float g = m->view.ice.g;
  m->fg.dom = m->view.geom.dom;
  m->fg.layer = m->view.ice.layer;
  m->fg.n_dom = m->view.geom.n_dom;
  m->fg.L = m->view.ice.L;
  m->fg.z_top = m->view.ice.z_top;
  m->fg.dz = m->view.ice.dz;
  m->fg.be_over_b = m->view.scatter_effective ? 1.0f - g : 1.0f;
  m->fg.theta_c = std::acos(m->view.run.cos_cherenkov);
  ppk::DeviceScope dev_scope(m->view.device);
  cudaError_t e = dev_scope.status();
  const size_t B = (size_t)max_batch, H = (size_t)kHid;
#define PP_A(x) \
  if (e == cudaSuccess) e = (x)
  PP_A(cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->view.device));
  if (e == cudaSuccess && m->sms < 1) e = cudaErrorInvalidDevice;
  PP_A(dalloc(&m->p, kNParams));
  PP_A(dalloc(&m->g, kNParams));
  PP_A(dalloc(&m->m, kNParams));
  PP_A(dalloc(&m->v, kNParams));
  PP_A(dalloc(&m->wb[0], H * kIn));
  for (int l = 1; l < kLayers; ++l) PP_A(dalloc(&m->wb[l], H * H));
  for (int l = 0; l < kLayers; ++l) {
    PP_A(dalloc(&m->z[l], B * H));
    PP_A(dalloc(&m->h[l], B * H));
    PP_A(dalloc(&m->dz[l], B * H));
  }
  PP_A(dalloc(&m->t1, B * H));
  PP_A(dalloc(&m->t2, B * H));
  PP_A(dalloc(&m->loss, 1));
  PP_A(dalloc(&m->err, 64));
  PP_A(dalloc(&m->wpack, packed_weight_bytes()));
  PP_A(dalloc(&m->wpack_bwd, packed_bwd_bytes()));
  PP_A(dalloc(&m->dw_part, (size_t)m->sms * kHid * kHid));
  PP_A(dalloc(&m->bfeat, B * kIn));
  PP_A(dalloc(&m->bnph, B));
  PP_A(dalloc(&m->bcnt, B));
  PP_A(dalloc(&m->head_part, (B / kHeadPartPairs) * kHeadPartCols));
  PP_A(dalloc(&m->head_lpart, B / kHeadPartPairs));
  PP_A(dalloc(&m->ice_cum, (size_t)m->fg.L));
  m->fg.cum = m->ice_cum;
  PP_A(launch_ice_cum(m->fg, m->ice_cum, 0));
  PP_A(cudaDeviceSynchronize());
  PP_A(dalloc(&m->ps, (size_t)max_rows));
  PP_A(dalloc(&m->pd, (size_t)max_rows));
  PP_A(dalloc(&m->count, 1));
  m->sprep_cap = m->fg.n_dom > 0 ? std::max<int64_t>(1, 8 * (max_rows / m->fg.n_dom)) : 1;
  PP_A(dalloc(&m->sprep, (size_t)m->sprep_cap));
  PP_A(cudaMemset(m->loss, 0, sizeof(double)));
  PP_A(cudaMemset(m->err, 0, 64 * sizeof(int)));
  PP_A(cudaMemset(m->p, 0, sizeof(float) * kNParams));
#undef PP_A
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    pp_mlp_destroy(m);
    return PP_ENOMEM;
  }
  *out = m;
  return PP_OK;
}

int pp_mlp_destroy(pp_mlp* m) {
  if (!m) return PP_OK;
  ppk::DeviceScope dev_scope(m->view.device);
  cudaDeviceSynchronize();
  void* bufs[] = {m->p,   m->g,     m->m,         m->v,  m->t1, m->t2,    m->loss, m->err,
                  m->wpack, m->wpack_bwd, m->ps, m->pd, m->count, m->ice_cum, m->dw_part,
                  m->head_part, m->head_lpart, m->pass_count, m->near_bcount, m->near_boff, m->bfeat,
                  m->bnph, m->bcnt, m->sprep};
  for (void* b : bufs) cudaFree(b);
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(m->wb[l]);
    cudaFree(m->z[l]);
    cudaFree(m->h[l]);
    cudaFree(m->dz[l]);
  }
  if (m->ctx) ppk::attach_server(m->ctx, -1);
  delete m;
  return PP_OK;
}

const char* pp_mlp_last_error(const pp_mlp* m) { return m ? m->last_error.c_str() : "null"; }

int pp_mlp_set_params(pp_mlp* m, const float* params, int64_t n) {
  if (!m || !params || n != kNParams) return PP_EINVAL;
  cudaStream_t st = m->view.stream;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  PP_MLP_CUDA(cudaMemcpyAsync(m->p, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, st));
  PP_MLP_CUDA(cudaMemsetAsync(m->m, 0, sizeof(float) * kNParams, st));
  PP_MLP_CUDA(cudaMemsetAsync(m->v, 0, sizeof(float) * kNParams, st));
  m->step = 0;
  m->weights_version += 1;
  int rc = refresh_bf16(m, st);
  if (rc) return rc;
  return mlp_sync(m, st);
}

int pp_mlp_get_params(pp_mlp* m, float* params, int64_t n) {
  if (!m || !params || n != kNParams) return PP_EINVAL;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  PP_MLP_CUDA(cudaStreamSynchronize(m->view.stream));
  PP_MLP_CUDA(cudaMemcpy(params, m->p, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  return PP_OK;
}

int pp_mlp_get_state(pp_mlp* m, float* params, float* m1, float* v1, int64_t n, int64_t* step) {
  if (!m || !params || n != kNParams) return PP_EINVAL;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  PP_MLP_CUDA(cudaStreamSynchronize(m->view.stream));
  PP_MLP_CUDA(cudaMemcpy(params, m->p, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  if (m1) PP_MLP_CUDA(cudaMemcpy(m1, m->m, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  if (v1) PP_MLP_CUDA(cudaMemcpy(v1, m->v, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  if (step) *step = m->step;
  return PP_OK;
}

int pp_mlp_set_state(pp_mlp* m, const float* params, const float* m1, const float* v1, int64_t n,
                     int64_t step) {
  if (!m || !params || n != kNParams || step < 0) return PP_EINVAL;
  for (int64_t i = 0; i < kNParams; ++i) {
    if (!std::isfinite(params[i]) || (m1 && !std::isfinite(m1[i])) ||
        (v1 && !(std::isfinite(v1[i]) && v1[i] >= 0.0f)))
      return mfail(m, PP_EINVAL, "non-finite parameter or moment, or negative second moment");
  }
  cudaStream_t st = m->view.stream;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  PP_MLP_CUDA(cudaMemcpyAsync(m->p, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, st));
  if (m1)
    PP_MLP_CUDA(cudaMemcpyAsync(m->m, m1, sizeof(float) * kNParams, cudaMemcpyHostToDevice, st));
  else
    PP_MLP_CUDA(cudaMemsetAsync(m->m, 0, sizeof(float) * kNParams, st));
  if (v1)
    PP_MLP_CUDA(cudaMemcpyAsync(m->v, v1, sizeof(float) * kNParams, cudaMemcpyHostToDevice, st));
  else
    PP_MLP_CUDA(cudaMemsetAsync(m->v, 0, sizeof(float) * kNParams, st));
  m->step = step;
  m->weights_version += 1;
  int rc = refresh_bf16(m, st);
  if (rc) return rc;
  return mlp_sync(m, st);
}

int pp_mlp_features(pp_mlp* m, const pp_source* d_src, const int32_t* d_pair_src,
                    const int32_t* d_pair_dom, int64_t n, uint16_t* d_feat, void* stream) {
  if (!m || n < 0 || (n > 0 && (!d_src || !d_pair_src || !d_pair_dom || !d_feat))) return PP_EINVAL;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : m->view.stream;
  PP_MLP_CUDA(launch_features(m->fg, d_src, d_pair_src, d_pair_dom, n,
                              reinterpret_cast<__nv_bfloat16*>(d_feat), st));
  return PP_OK;
}

int pp_mlp_forward(pp_mlp* m, const uint16_t* d_feat, const float* d_nph, int64_t n,
                   float* d_lambda, void* stream) {
  ppk::NvtxRange range("pp.mlp.forward");
  if (!m || n < 0 || (n > 0 && (!d_feat || !d_nph || !d_lambda))) return PP_EINVAL;
  if (n > 0 && !aligned16(d_feat)) return mfail(m, PP_EINVAL, "features must be 16-byte aligned");
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : m->view.stream;
  int rc;
  if ((rc = ensure_packed(m, st)) || (rc = ensure_hbias(m, st))) return rc;
  FusedArgs a = fused_args(m);
  a.feat = reinterpret_cast<const __nv_bfloat16*>(d_feat);
  a.n = n;
  a.nph = d_nph;
  a.lambda = d_lambda;
  PP_MLP_CUDA(launch_mlp_fused(a, &m->hbias, false, m->sms, st));
  return PP_OK;
}

int pp_mlp_gradients(pp_mlp* m, const uint16_t* d_feat, const float* d_nph, const float* d_count,
                     int64_t n, float* h_grads, double* h_loss) {
  if (!m || !d_feat || !d_nph || !d_count || !h_grads) return PP_EINVAL;
  int rc;
  if ((rc = check_batch(m, n, d_feat))) return rc;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = m->view.stream;
  PP_MLP_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), st));
  if ((rc = forward_backward(m, reinterpret_cast<const __nv_bfloat16*>(d_feat), d_nph, d_count,
                             (int)n, st)))
    return rc;
  if ((rc = mlp_sync(m, st))) return rc;
  PP_MLP_CUDA(cudaMemcpy(h_grads, m->g, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  if (h_loss) PP_MLP_CUDA(cudaMemcpy(h_loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
  return PP_OK;
}

int pp_mlp_train_step(pp_mlp* m, const uint16_t* d_feat, const float* d_nph, const float* d_count,
                      int64_t n, float lr, void* stream) {
  if (!m || !d_feat || !d_nph || !d_count || !(lr > 0.0f)) return PP_EINVAL;
  int rc;
  if ((rc = check_batch(m, n, d_feat))) return rc;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : m->view.stream;
  return train_step(m, reinterpret_cast<const __nv_bfloat16*>(d_feat), d_nph, d_count, n, lr, st);
}

int pp_mlp_train_step_rows(pp_mlp* m, const uint16_t* d_feat, const float* d_nph,
                           const float* d_count, int64_t n_rows, const int64_t* d_rows, int64_t n,
                           float lr, void* stream) {
  if (!m || !d_feat || !d_nph || !d_count || !d_rows || n_rows < 1 || !(lr > 0.0f))
    return PP_EINVAL;
  int rc;
  if ((rc = check_batch(m, n, d_feat))) return rc;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : m->view.stream;
  PP_MLP_CUDA(launch_gather_rows(reinterpret_cast<const __nv_bfloat16*>(d_feat), d_nph, d_count,
                                 n_rows, d_rows, n, m->bfeat, m->bnph, m->bcnt, m->err, st));
  return train_step(m, m->bfeat, m->bnph, m->bcnt, n, lr, st);
}

}  // extern "C"

namespace {

int train_step(pp_mlp* m, const __nv_bfloat16* feat, const float* nph, const float* cnt,
               int64_t n, float lr, cudaStream_t st) {
  ppk::NvtxRange range("pp.mlp.train_step");
  int rc;
  if ((rc = forward_backward(m, feat, nph, cnt, (int)n, st))) return rc;
  m->step += 1;
  m->weights_version += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.0f - (float)std::pow(0.9, (double)m->step);
  const float bc2 = 1.0f - (float)std::pow(0.999, (double)m->step);
  // Adam on each weight block (writing its BF16 copy) and on the rest
  PP_MLP_CUDA(launch_adam(m->p + kOffW1, m->g + kOffW1, m->m + kOffW1, m->v + kOffW1,
                          (int64_t)kHid * kIn, lr, b1, b2, 1e-8f, bc1, bc2, m->wb[0], st));
  PP_MLP_CUDA(launch_adam(m->p + kOffB1, m->g + kOffB1, m->m + kOffB1, m->v + kOffB1, kHid, lr,
                          b1, b2, 1e-8f, bc1, bc2, nullptr, st));
  for (int l = 1; l < kLayers; ++l) {
    const int64_t o = off_w(l);
    PP_MLP_CUDA(launch_adam(m->p + o, m->g + o, m->m + o, m->v + o, (int64_t)kHid * kHid, lr, b1,
                            b2, 1e-8f, bc1, bc2, m->wb[l], st));
    const int64_t ob = off_b(l);
    PP_MLP_CUDA(launch_adam(m->p + ob, m->g + ob, m->m + ob, m->v + ob, kHid, lr, b1, b2, 1e-8f,
                            bc1, bc2, nullptr, st));
  }
  PP_MLP_CUDA(launch_adam(m->p + kOffW5, m->g + kOffW5, m->m + kOffW5, m->v + kOffW5, kHid + 1,
                          lr, b1, b2, 1e-8f, bc1, bc2, nullptr, st));
  return PP_OK;
}

}  // namespace

extern "C" {

int pp_mlp_loss(pp_mlp* m, double* loss) {
  if (!m || !loss) return PP_EINVAL;
  int rc;
  if ((rc = mlp_sync(m, m->view.stream))) return rc;
  PP_MLP_CUDA(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
  PP_MLP_CUDA(cudaMemset(m->loss, 0, sizeof(double)));
  return PP_OK;
}

int pp_mlp_dom_sums(pp_mlp* m, const pp_source* d_src, int64_t n_src, const float* d_nph_src,
                    float r_max, double* d_dom_sums, float* d_lambda, void* stream) {
  ppk::NvtxRange range("pp.mlp.dom_sums");
  if (!m || n_src < 0 || (n_src > 0 && (!d_src || !d_nph_src)) || (!d_dom_sums && !d_lambda) ||
      !(r_max > 0.0f))
    return PP_EINVAL;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : m->view.stream;
  const int n_dom = m->fg.n_dom;
  if (d_dom_sums) PP_MLP_CUDA(cudaMemsetAsync(d_dom_sums, 0, sizeof(double) * n_dom, st));
  if (d_lambda)
    PP_MLP_CUDA(cudaMemsetAsync(d_lambda, 0, sizeof(float) * (size_t)n_src * n_dom, st));
  if (n_dom == 0 || n_src == 0) return PP_OK;
  int rc;
  if ((rc = ensure_packed(m, st)) || (rc = ensure_hbias(m, st))) return rc;
  // pairs within r_max only: the network is evaluated on a compacted list,
  // in passes of `per` sources, whose candidate pairs (sources x DOMs) are 8
  // times what the buffers hold: at most an eighth are expected within r_max
  int64_t per = 8 * (m->max_rows / n_dom);
  if (per < 1) per = 1;
  // every pair of the call fits the buffers: one pass, no count to check, no wait
  const bool fits = n_src <= m->max_rows / n_dom;
  if (fits) per = n_src;
  // one pass: the pair search over sources s0 .. s0 + ns, then the network on
  // its pairs -- n of them, or (n_dev set) as many as the search counted
  auto run_pass = [&](int64_t s0, int64_t ns, int64_t n, const unsigned long long* n_dev) -> int {
    FusedArgs a = fused_args(m);
    a.src = d_src;
    if (ns <= m->sprep_cap) {  // the sources' part of the features, once per source
      PP_MLP_CUDA(launch_src_prep(m->fg, d_src, s0, ns, m->sprep, st));
      a.sprep = m->sprep;
      a.sprep_base = s0;
    }
    a.ps = m->ps;
    a.pd = m->pd;
    a.n = n;
    a.n_dev = n_dev;
    a.nph = d_nph_src;
    a.dom_sum = d_dom_sums;
    a.lambda_out = d_lambda;
    PP_MLP_CUDA(launch_mlp_fused(a, &m->hbias, true, m->sms, st));
    return PP_OK;
  };
  // First every pass is enqueued at once, the network reading its row count
  // from the search's count in device memory; the host waits once, at the
  // end, for the passes' counts.  Only if some pass found more pairs than the
  // buffers hold does the call start over, pass by pass, waiting for each
  // count and passing fewer sources at a time where needed.
  const int64_t n_pass = (n_src + per - 1) / per;
  if (n_pass > m->pass_cap) {
    cudaFree(m->pass_count);
    m->pass_count = nullptr;
    m->pass_cap = 0;
    PP_MLP_CUDA(dalloc(&m->pass_count, (size_t)n_pass));
    m->pass_cap = n_pass;
  }
  for (int64_t k = 0; k < n_pass; ++k) {
    const int64_t s0 = k * per, ns = std::min(per, n_src - s0);
    PP_MLP_CUDA(cudaMemsetAsync(m->count, 0, sizeof(unsigned long long), st));
    PP_MLP_CUDA(launch_near_pairs(m->fg, d_src, s0, ns, r_max, m->max_rows, m->ps, m->pd,
                                  m->count, st));
    PP_MLP_CUDA(cudaMemcpyAsync(m->pass_count + k, m->count, sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, st));
    if ((rc = run_pass(s0, ns, m->max_rows, m->count))) return rc;
  }
  if (fits) return PP_OK;
  std::vector<unsigned long long> counts((size_t)n_pass);
  PP_MLP_CUDA(cudaMemcpyAsync(counts.data(), m->pass_count, sizeof(unsigned long long) * n_pass,
                              cudaMemcpyDeviceToHost, st));
  PP_MLP_CUDA(cudaStreamSynchronize(st));
  bool overflow = false;
  for (unsigned long long c : counts) overflow |= (int64_t)c > m->max_rows;
  if (!overflow) return PP_OK;
  if (d_dom_sums) PP_MLP_CUDA(cudaMemsetAsync(d_dom_sums, 0, sizeof(double) * n_dom, st));
  if (d_lambda)
    PP_MLP_CUDA(cudaMemsetAsync(d_lambda, 0, sizeof(float) * (size_t)n_src * n_dom, st));
  for (int64_t s0 = 0; s0 < n_src;) {
    int64_t ns = (n_src - s0) < per ? (n_src - s0) : per;
    unsigned long long cnt = 0;
    for (;;) {
      PP_MLP_CUDA(cudaMemsetAsync(m->count, 0, sizeof(unsigned long long), st));
      PP_MLP_CUDA(launch_near_pairs(m->fg, d_src, s0, ns, r_max, m->max_rows, m->ps, m->pd,
                                    m->count, st));
      PP_MLP_CUDA(cudaMemcpyAsync(&cnt, m->count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
      PP_MLP_CUDA(cudaStreamSynchronize(st));
      if ((int64_t)cnt <= m->max_rows || ns == 1) break;
      ns = (ns + 1) / 2;  // too many close pairs for the buffers: fewer sources
    }
    if ((int64_t)cnt > m->max_rows)
      return mfail(m, PP_EINVAL, "one source has more pairs within r_max than max_rows");
    if (cnt > 0 && (rc = run_pass(s0, ns, (int64_t)cnt, nullptr))) return rc;
    s0 += ns;
  }
  return PP_OK;
}

int pp_mlp_near_pairs(pp_mlp* m, const pp_source* d_src, int64_t n_src, float r_max,
                      int64_t max_out, int32_t* d_pair_src, int32_t* d_pair_dom,
                      uint64_t* h_count) {
  if (!m || n_src < 0 || (n_src > 0 && !d_src) || !h_count || max_out < 0 || !(r_max > 0.0f) ||
      (max_out > 0 && (!d_pair_src || !d_pair_dom)))
    return PP_EINVAL;
  ppk::DeviceScope dev_scope(m->view.device);
  PP_MLP_CUDA(dev_scope.status());
  cudaStream_t st = m->view.stream;
  const int64_t nb = near_pairs_ordered_blocks(n_src * (int64_t)m->fg.n_dom);
  if (nb > m->near_cap) {
    PP_MLP_CUDA(cudaStreamSynchronize(st));
    cudaFree(m->near_bcount);
    cudaFree(m->near_boff);
    m->near_bcount = nullptr;
    m->near_boff = nullptr;
    m->near_cap = 0;
    if (dalloc(&m->near_bcount, (size_t)nb) != cudaSuccess ||
        dalloc(&m->near_boff, (size_t)nb) != cudaSuccess) {
      (void)cudaGetLastError();
      return mfail(m, PP_ENOMEM, "pair search scratch");
    }
    m->near_cap = nb;
  }
  PP_MLP_CUDA(cudaMemsetAsync(m->count, 0, sizeof(unsigned long long), st));
  PP_MLP_CUDA(launch_near_pairs_ordered(m->fg, d_src, n_src, r_max, max_out, d_pair_src,
                                        d_pair_dom, m->count, m->near_bcount, m->near_boff, st));
  unsigned long long c = 0;
  PP_MLP_CUDA(cudaMemcpyAsync(&c, m->count, sizeof(c), cudaMemcpyDeviceToHost, st));
  PP_MLP_CUDA(cudaStreamSynchronize(st));
  *h_count = c;
  return PP_OK;
}

int pp_mlp_set_activation(pp_mlp* m, int32_t act) {
  if (!m || (act != PP_MLP_ACT_SILU && act != PP_MLP_ACT_HARD_SWISH)) return PP_EINVAL;
  static_assert(PP_MLP_ACT_SILU == kActSilu && PP_MLP_ACT_HARD_SWISH == kActHardSwish, "codes");
  m->act = act;
  return PP_OK;
}

int pp_mlp_set_exact_silu(pp_mlp* m, int exact) {
  if (!m) return PP_EINVAL;
  m->exact_silu = exact ? 1 : 0;
  return PP_OK;
}

int pp_mlp_sync(pp_mlp* m) {
  if (!m) return PP_EINVAL;
  return mlp_sync(m, m->view.stream);
}

}  // extern "C"
