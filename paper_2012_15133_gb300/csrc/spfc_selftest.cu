// Self-test of the device-side bounded wait used by the grid barrier of the
// fused column pass (declared in include/spfc.h).
#include <cuda_runtime.h>

#include "../../include/spfc.h"
#include "spfc_kernels2d.cuh"

namespace {

// One thread waits (bounded) until *ctr >= target; nothing advances the
// counter, so the wait ends by its limit unless target <= *ctr already.
__global__ void k_wait_selftest(const unsigned long long* ctr, unsigned long long target, long long polls,
                                int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *status = spfc::wait_counter(ctr, target, polls) ? (int)spfc::DEV_OK : (int)spfc::DEV_TIMEOUT;
}

}  // namespace

extern "C" int spfc_wait_selftest(unsigned long long target, long long polls, void* cuda_stream) {
  if (polls < 0 || polls > (1ll << 24)) return SPFC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long* ctr = nullptr;
  int* status = nullptr;
  if (cudaMalloc(&ctr, sizeof(unsigned long long)) != cudaSuccess) return SPFC_ENOMEM;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(ctr);
    return SPFC_ENOMEM;
  }
  int host = -1;
  cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0xff, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(ctr, target, polls, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ctr);
  cudaFree(status);
  if (e != cudaSuccess) return SPFC_ECUDA;
  if (host == (int)spfc::DEV_TIMEOUT) return SPFC_ETIMEOUT;
  return host == (int)spfc::DEV_OK ? SPFC_OK : SPFC_ECUDA;
}
