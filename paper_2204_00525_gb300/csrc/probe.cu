// Measurement aid (not part of the paper's method): the FP64 FMA issue rate of this GPU,
// the ceiling of the FP64-pipe-bound kernels (the TSQR leaves, the FP64 scans).  Every
// thread runs eight independent FMA chains, so the rate is the pipe's throughput, not a
// dependent chain's latency; 152 x 8 blocks of 256 threads keep 64 warps on every SM.
#include "kernels.cuh"

namespace fig {

static __device__ double g_fma_sink;

constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma_rate(int iters, double seed) {
  double a[kFmaChains];
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) a[c] = seed + 1e-9 * (threadIdx.x + 37 * c);
  const double b = 0.9999999, d = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) s += a[c];
  if (s == -1.0) g_fma_sink = s;   // never true for these inputs; keeps the chains live
}

}  // namespace fig

extern "C" int figaro_fp64_fma_rate(double* tflops, void* stream) {
  using namespace fig;
  if (!tflops) return FIGARO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FIGARO_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FIGARO_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 8192;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FIGARO_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FIGARO_ERR_CUDA;
  }
  k_fp64_fma_rate<<<blocks, threads, 0, st>>>(iters, 1.0);   // warm-up
  cudaEventRecord(e0, st);
  for (int r = 0; r < 5; ++r) k_fp64_fma_rate<<<blocks, threads, 0, st>>>(iters, 1.0 + r);
  cudaEventRecord(e1, st);
  int rc = FIGARO_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess)
    rc = FIGARO_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != FIGARO_OK) return rc;
  const double flops = 5.0 * blocks * threads * (double)iters * kFmaChains * 2.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return FIGARO_OK;
}
