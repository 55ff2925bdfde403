// Measured FP64 arithmetic peak of the device (the denominator of the FP64-pipe roofline of the
// trace kernels).  Not part of the method: a calibration kernel.
//
// Every thread runs kChains independent chains of fused multiply-adds x <- x * a + b (a slightly
// below 1, so the values stay bounded), which keeps each SM's FP64 units busy without memory
// traffic.  The rate is FMA lane-operations per second over a launch of num_SMs x blocks, timed
// with CUDA events on the caller's stream; the best of `repeats` launches is returned.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mt.h"

namespace {

constexpr int kProbeBlock = 256;
constexpr int kChains = 8;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(kProbeBlock) fp64_fma_kernel(int64_t iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) g_probe_sink = s;  // keeps the chains live (the values stay near 0.1)
}

}  // namespace

extern "C" mt_status mt_probe_fp64_fma_rate(int64_t iters, int32_t repeats, double* fma_per_s, void* stream_) {
  if (!fma_per_s || iters < 1 || repeats < 1) return MT_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  int dev = 0, sms = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MT_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MT_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fp64_fma_kernel, kProbeBlock, 0) != cudaSuccess || bps < 1)
    bps = 1;
  const int grid = sms * bps;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MT_ERR_CUDA;
  double best = 0.0;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {  // launch 0 warms up
    e = cudaEventRecord(e0, stream);
    if (e == cudaSuccess) {
      fp64_fma_kernel<<<grid, kProbeBlock, 0, stream>>>(iters, 0.999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0.0f) {
      const double ops = (double)grid * kProbeBlock * (double)kChains * (double)iters;
      const double rate = ops / (ms * 1e-3);
      if (rate > best) best = rate;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return MT_ERR_CUDA;
  *fma_per_s = best;
  return MT_OK;
}
