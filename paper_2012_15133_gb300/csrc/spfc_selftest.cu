// Self-test of the device-side bounded waits used by the grid barriers of
// the fused column pass and of the persistent step (declared in
// include/spfc.h).
#include <cuda_runtime.h>

#include "../../include/spfc.h"
#include "spfc_step2d_persist.cuh"

namespace {

// One thread runs both bounded waits (the fused column pass's, then the
// persistent step's acquire polls) until *ctr >= target; nothing advances the
// counter, so each ends by its limit unless target <= *ctr already. Both give
// the same answer, or the status reports the disagreement (-1).
__global__ void k_wait_selftest(const unsigned long long* ctr, unsigned long long target, long long polls,
                                int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const bool a = spfc::wait_counter(ctr, target, polls);
    const bool b = spfc::wait_counter_acquire(ctr, target, polls);
    *status = (a != b) ? -1 : (a ? (int)spfc::DEV_OK : (int)spfc::DEV_TIMEOUT);
  }
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

// ---------------------------------------------------------------------------
// Measured float64 FMA rate of the device (the arithmetic roofline of the
// float64 step): every thread runs kChains independent chains of `iters`
// float64 fused multiply-adds (no dependence between chains, so the FP64
// pipe, not latency, sets the time), on an SM-count multiple of blocks.
// ---------------------------------------------------------------------------
namespace {
constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma_rate(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-3 * threadIdx.x + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}
}  // namespace

extern "C" int spfc_fp64_fma_rate(double* gflops, void* cuda_stream) {
  if (!gflops) return SPFC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPFC_ECUDA;
  const int threads = 256, blocks = 4 * nsm, iters = 4096;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return SPFC_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_dfma_rate<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || !(best > 0.f)) return SPFC_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * threads;
  *gflops = flops / (best * 1e-3) / 1e9;
  return SPFC_OK;
}
