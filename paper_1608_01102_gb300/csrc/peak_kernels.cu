// FP32 FMA throughput probe of the device: the denominator of the ALU-side
// roofline of the SCGS smoother, whose dense 5x5 / 7x7 block arithmetic puts
// it near the FP32 CUDA-core ridge.  Measurement support only; no step of the
// method runs here.
#include <cuda_runtime.h>

#include "../../include/stc.h"
#include "stc_internal.cuh"
#include "stc_kernels.h"

namespace stc {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;      // independent FMA chains per thread (hides the FMA latency)
constexpr int kPeakIters = 2048;    // loop trips; each trip issues kPeakChains * 4 FMAs

// result sink: one float per CTA, so the chains are not optimised away
static __device__ float g_peak_sink[4096];

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float seed, float m) {
  float a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed + 0.001f * (float)(threadIdx.x + c);
  const float b = 0.999f;
  for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = fmaf(a[c], b, m);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += a[c];
  if (s == 12345.678f) g_peak_sink[blockIdx.x & 4095] = s;   // practically never stored
}

}  // namespace
}  // namespace stc

extern "C" stc_status stc_measure_fp32_peak(void* cuda_stream, double* gflops) {
  using namespace stc;
  if (!gflops) {
    set_last_error("stc_measure_fp32_peak: null argument");
    return STC_ERR_INVALID_ARG;
  }
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel, kPeakThreads, 0);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;   // four full waves
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(t0, st);
    if (e == cudaSuccess) {
      fma_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(1.0f, 1e-3f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0 && ms > 0.f) {   // the first launch warms up
      const float r = 2.0f * kPeakChains * 4.0f * kPeakIters * (float)kPeakThreads * (float)blocks / (ms * 1e-3f);
      if (r > best) best = r;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return STC_ERR_CUDA;
  }
  *gflops = best * 1e-9;
  return STC_OK;
}
