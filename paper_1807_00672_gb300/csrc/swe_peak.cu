// Measurement helper (no counterpart in the paper): FP64 fused multiply-add
// throughput of the current device. The FP64 step is bound by FP64
// arithmetic on GB300, so bench.py reports it against this measured rate
// (and against the nominal rate) as well as against HBM bandwidth.
#include <cuda_runtime.h>

#include "../../include/swe.h"

namespace {

constexpr int kChains = 8;    // independent DFMA chains per thread
constexpr int kThreads = 256;

// Each thread runs kChains independent chains x <- x a + b for `iters`
// iterations (values stay bounded for |a| < 1). The sum is stored only if it
// equals `never`, which it does not, so the chains cannot be removed.
__global__ void __launch_bounds__(kThreads) k_dfma_rate(double* out, int iters, double a, double b,
                                                       double never) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x + 1) * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == never) out[blockIdx.x] = s;
}

}  // namespace

extern "C" swe_status swe_fp64_fma_rate(void* cuda_stream, double* tflops) {
  if (!tflops) return SWE_EINVAL;
  *tflops = 0.0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dfma_rate, kThreads, 0) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return SWE_ECUDA;
  }
  const int blocks = sms * occ;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  swe_status rc = SWE_OK;
  if (cudaMalloc((void**)&out, sizeof(double) * blocks) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = SWE_ECUDA;
  } else {
    const int iters = 4096;
    k_dfma_rate<<<blocks, kThreads, 0, st>>>(out, 64, 0.999999, 1e-7, -1.0);  // warm-up
    cudaEventRecord(e0, st);
    k_dfma_rate<<<blocks, kThreads, 0, st>>>(out, iters, 0.999999, 1e-7, -1.0);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        !(ms > 0.0f)) {
      rc = SWE_ECUDA;
    } else {
      const double flops = 2.0 * kChains * (double)iters * kThreads * (double)blocks;
      *tflops = flops / (ms * 1e-3) / 1e12;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (rc != SWE_OK) cudaGetLastError();
  return rc;
}
