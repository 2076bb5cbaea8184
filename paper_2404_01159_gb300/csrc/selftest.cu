// Failure-detection self-test of the bounded device waits.
//
// The reproduction and association kernels wait on mbarriers for their TMA
// copies with a poll limit; a wait that runs out sets a status word that the
// host reads (RVEA_ERR_TIMEOUT) instead of hanging the GPU.  This kernel runs
// the same wait on a barrier that nothing arrives at, so the limit is always
// reached: the test that the mechanism ends and reports, without a fault or
// a hang.
#include <cuda_runtime.h>

#include "../../include/rvea.h"
#include "rvea_device.cuh"

namespace rvea {

static __device__ int g_selftest_status;   // 1: the wait completed, 2: it gave up

__global__ void k_selftest_wait(uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);   // one arrival expected; none comes
  fence_mbar_init();
  g_selftest_status = mbar_wait(&bar, 0u, polls) ? 1 : 2;
}

}  // namespace rvea

using namespace rvea;

extern "C" rvea_status rvea_selftest_wait(int polls, void *cuda_stream) {
  if (polls < 1 || polls > (1 << 20)) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_selftest_status, &zero, sizeof(int), 0,
                              cudaMemcpyHostToDevice, st) != cudaSuccess)
    return RVEA_ERR_CUDA;
  k_selftest_wait<<<1, 32, 0, st>>>((uint32_t)polls);
  if (cudaGetLastError() != cudaSuccess) return RVEA_ERR_CUDA;
  int s = 0;
  if (cudaMemcpyFromSymbolAsync(&s, g_selftest_status, sizeof(int), 0,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RVEA_ERR_CUDA;
  return s == 2 ? RVEA_ERR_TIMEOUT : (s == 1 ? RVEA_OK : RVEA_ERR_CUDA);
}
