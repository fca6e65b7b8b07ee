// Measurement support (not part of the method): the FP64 fused-multiply-add throughput of the
// device, measured with a kernel of independent FMA chains, as the roofline denominator of the
// FP64-bound kernels.
#include <cuda_runtime.h>

#include "spadj.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread (hide the FMA latency)

// Every thread runs kChains chains of `iters` FMAs, a <- a * m + c with |m| < 1 so the values stay
// bounded; the result is stored only if it equals a value it never takes, which keeps the chains
// live without a store per thread.
__global__ void __launch_bounds__(256) dfma_probe_kernel(int iters, double m, double c, double* sink) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" spadj_status spadj_fp64_peak(void* cuda_stream, int iters, double* gflops_host, double* ms_host) {
  if (!gflops_host || iters < 1) return SPADJ_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPADJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPADJ_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_probe_kernel, 256, 0) != cudaSuccess)
    return SPADJ_ERR_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return SPADJ_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_probe_kernel<<<blocks, 256, 0, st>>>(iters / 10 + 1, 0.999999, 1e-6, sink);  // warm-up
  cudaEventRecord(e0, st);
  dfma_probe_kernel<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-6, sink);
  cudaEventRecord(e1, st);
  spadj_status res = SPADJ_OK;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    res = SPADJ_ERR_CUDA;
  } else {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * (double)iters * 256.0 * blocks;
    *gflops_host = flops / (ms * 1e-3) / 1e9;
    if (ms_host) *ms_host = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return res;
}
