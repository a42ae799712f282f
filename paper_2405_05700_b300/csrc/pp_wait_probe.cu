// pp_debug_wait_timeout: the bounded mbarrier wait of the tensor-core kernels
// (tc::mbar_wait) on a barrier that nothing completes.  The wait gives up at
// its time limit and the kernel reports it, so a lost arrival ends as an error
// status the host reads, never as a hung GPU; the test of that path runs this.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pp.h"
#include "pp_internal.h"
#include "tc_gemm.cuh"

namespace {

__global__ void k_wait_nothing(uint64_t limit_ns, int* timed_out, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);  // one arrival expected; none comes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = tc::globaltimer_ns();
    const bool done = tc::mbar_wait(&bar, 0, 0xffffffffu, limit_ns);
    *waited_ns = tc::globaltimer_ns() - t0;
    *timed_out = done ? 0 : 1;
  }
}

}  // namespace

extern "C" int pp_debug_wait_timeout(int32_t device, uint64_t limit_ns, int32_t* timed_out,
                                     uint64_t* waited_ns) {
  if (!timed_out || !waited_ns || limit_ns < 1000ull || limit_ns > 1000000000ull) return PP_EINVAL;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) return PP_ENODEV;
  if (device < 0 || device >= n_dev) return PP_EINVAL;
  ppk::DeviceScope dev_scope(device);
  if (dev_scope.status() != cudaSuccess) return PP_ECUDA;
  int* d_flag = nullptr;
  unsigned long long* d_ns = nullptr;
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) return PP_ENOMEM;
  if (cudaMalloc(&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(d_flag);
    return PP_ENOMEM;
  }
  int rc = PP_OK;
  k_wait_nothing<<<1, 32>>>(limit_ns, d_flag, d_ns);
  int flag = 0;
  unsigned long long ns = 0;
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = PP_ECUDA;
  cudaFree(d_flag);
  cudaFree(d_ns);
  if (rc == PP_OK) {
    *timed_out = flag;
    *waited_ns = ns;
  }
  return rc;
}
