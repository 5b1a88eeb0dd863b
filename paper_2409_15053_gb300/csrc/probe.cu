// Measured arithmetic peaks of the GPU the library runs on: the denominators
// of the filter kernels' ALU fractions. A grid of 8 resident CTAs per SM runs
// independent multiply-add chains (eight per thread, so the pipe, not the
// dependency latency, sets the rate) and is timed with CUDA events.
#include "flz_internal.h"

namespace flz {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// FP64: a = a * x + y per chain and iteration (one FMA = 2 flops)
__global__ void __launch_bounds__(kThreads) fp64_fma_loop(int iters, double x, double y, double* out) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) out[0] = s;  // keeps the chains live
}

// 32-bit integer multiply-add (the operation of the fixed-point filter's limb
// products): a = a * x + y per chain and iteration
__global__ void __launch_bounds__(kThreads) int_mad_loop(int iters, uint32_t x, uint32_t y, uint32_t* out) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 7u + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = a[c] * x + y;
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0x9e3779b9u) out[0] = s;
}

}  // namespace

double measure_alu_peak(int kind) {
  int dev = 0, sms = 0;
  FLZ_CUDA(cudaGetDevice(&dev));
  FLZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * 8;
  const int iters = kind == 0 ? 4096 : 65536;
  DevBuf<double> d;
  d.reserve(1);
  cudaEvent_t e0, e1;
  FLZ_CUDA(cudaEventCreate(&e0));
  FLZ_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first run is a warm-up; the fastest of the rest counts
    FLZ_CUDA(cudaEventRecord(e0));
    if (kind == 0)
      fp64_fma_loop<<<grid, kThreads>>>(iters, 0.999999, 1e-9, d.p);
    else
      int_mad_loop<<<grid, kThreads>>>(iters, 2654435761u, 12345u, reinterpret_cast<uint32_t*>(d.p));
    FLZ_LAUNCH_CHECK();
    FLZ_CUDA(cudaEventRecord(e1));
    FLZ_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FLZ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double ops = (double)grid * kThreads * kChains * (double)iters;  // multiply-adds
  return 2.0 * ops / (best * 1e-3);                                      // flops (or integer ops) per second
}

}  // namespace flz
