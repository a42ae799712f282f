// pp_measure_issue_rate: measured FP32 and SFU lane-operation rates of the
// device, the denominators for the propagation kernel's pipe utilisation.
//
// Each thread runs kChains independent dependency chains so that the pipe,
// not the instruction latency, sets the rate; the grid fills every SM to the
// maximum of resident threads.  One lane operation = one FMA (FP32 kernel) or
// one lg2.approx (SFU kernel), the convention of the propagation's per-step
// counts (an FMA counts once).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pp.h"
#include "pp_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 16;

// x <- x * b + c on every chain; with 0 < b < 1 the chains converge to
// c / (1 - b), so the final sum is finite and the store below never happens
// for the arguments the host passes.  The condition keeps the chains live.
__global__ void __launch_bounds__(kThreads) k_issue_fma(float b, float c, int iters, float* sink) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (float)threadIdx.x + (float)j;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == -1.0f) sink[0] = s;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x <- log2(x) + c: for c = 2 the chains converge to the fixed point x = 4
// (slope 1 / (4 ln 2) < 1), so every argument stays positive and normal.
__global__ void __launch_bounds__(kThreads) k_issue_sfu(float c, int iters, float* sink) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 3.0f + 1e-3f * (float)(threadIdx.x + j);
#pragma unroll 2
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = lg2_approx(x[j]) + c;
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == -1.0f) sink[0] = s;
}

}  // namespace

extern "C" int pp_measure_issue_rate(int32_t device, int32_t kind, double* lane_ops_per_s,
                                     double* ms) {
  if ((kind != PP_ISSUE_FP32_FMA && kind != PP_ISSUE_SFU_LG2) || !lane_ops_per_s)
    return PP_EINVAL;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) return PP_ENODEV;
  if (device < 0 || device >= n_dev) return PP_EINVAL;
  ppk::DeviceScope dev_scope(device);
  if (dev_scope.status() != cudaSuccess) return PP_ECUDA;
  int sms = 0, max_threads = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, device) !=
          cudaSuccess)
    return PP_ECUDA;
  const int blocks = sms * (max_threads / kThreads);
  // about 30 ms per launch at the nominal rates (FMA 128, SFU 16 lanes per SM and clock)
  const int iters = kind == PP_ISSUE_FP32_FMA ? 200000 : 25000;

  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  int rc = PP_OK;
  float t_ms = 0.f;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return PP_ENOMEM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = PP_ECUDA;
  } else {
    for (int rep = 0; rep < 2 && rc == PP_OK; ++rep) {  // rep 0: warm-up
      cudaEventRecord(e0, st);
      if (kind == PP_ISSUE_FP32_FMA)
        k_issue_fma<<<blocks, kThreads, 0, st>>>(0.999f, 1e-3f, iters, sink);
      else
        k_issue_sfu<<<blocks, kThreads, 0, st>>>(2.0f, iters, sink);
      cudaEventRecord(e1, st);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess)
        rc = PP_ECUDA;
    }
  }
  if (rc == PP_OK) {
    const double ops = (double)blocks * kThreads * (double)iters * kChains;
    *lane_ops_per_s = ops / (t_ms * 1e-3);
    if (ms) *ms = t_ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(sink);
  return rc;
}
