// kde_probe.cu -- microbenchmarks of the three pipes the pair kernels use:
// FP32 FMA, MUFU ex2 and FP64 FMA.  Each kernel runs 8 independent dependency
// chains per thread with every block resident at once and is timed with CUDA
// events; the result is operations per second per SM (divide by the SM clock
// sampled meanwhile to get operations per clock).  The numbers size the
// ALU roofline of the pair kernels (their per-pair instruction mix is fixed).
#include "kde_internal.cuh"

#include <algorithm>
#include <vector>

namespace kde {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 8192;
constexpr int kThreads = 256;

__device__ __forceinline__ float ex2_probe(float t) {
  float e;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(t));
  return e;
}

__global__ void __launch_bounds__(kThreads) probe_fma32(float* sink, long long* cyc, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * threadIdx.x + k;
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678f) sink[0] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) probe_ex2(float* sink, long long* cyc) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 0.25f + 0.01f * k + 1e-5f * threadIdx.x;
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = ex2_probe(-a[k]);   // stays in [0.5, 1)
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678f) sink[0] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kThreads) probe_fma64(double* sink, long long* cyc, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * threadIdx.x + k;
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 2
  for (int i = 0; i < kIters / 8; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678) sink[0] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace kde

using namespace kde;

extern "C" kde_status kde_probe_pipe_rates(double* out, int cap) {
  if (!out || cap < 5) return set_err(KDE_ERR_INVALID, "need room for 5 values");
  const int sms = num_sms();
  void* sink = nullptr;
  long long* cyc = nullptr;
  const int max_grid = sms * (2048 / kThreads);
  if (cudaMalloc(&sink, 64) != cudaSuccess || cudaMalloc(&cyc, sizeof(long long) * max_grid) != cudaSuccess) {
    cudaGetLastError();
    if (sink) cudaFree(sink);
    return set_err(KDE_ERR_OOM, "probe buffers");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<long long> h(max_grid);
  double rates[3] = {0, 0, 0}, ticks_per_s = 0.0;
  for (int which = 0; which < 3; ++which) {
    // every block resident at once: grid = SMs x resident blocks per SM
    int per_sm = 0;
    if (which == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_fma32, kThreads, 0);
    if (which == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_ex2, kThreads, 0);
    if (which == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_fma64, kThreads, 0);
    per_sm = std::max(1, std::min(per_sm, 2048 / kThreads));
    const int grid = sms * per_sm;
    double ms_best = 1e30, cyc_best = 0;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0);
      if (which == 0) probe_fma32<<<grid, kThreads>>>(static_cast<float*>(sink), cyc, 0.999f, 1e-3f);
      if (which == 1) probe_ex2<<<grid, kThreads>>>(static_cast<float*>(sink), cyc);
      if (which == 2) probe_fma64<<<grid, kThreads>>>(static_cast<double*>(sink), cyc, 0.999, 1e-3);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaMemcpy(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
      std::vector<long long> sorted(h.begin(), h.begin() + grid);
      std::sort(sorted.begin(), sorted.end());
      if (ms < ms_best) {
        ms_best = ms;
        cyc_best = static_cast<double>(sorted[sorted.size() / 2]);
      }
    }
    const double iters = which == 2 ? kIters / 8 : kIters;
    const double ops_per_sm = static_cast<double>(per_sm) * kThreads * kChains * iters;
    rates[which] = ops_per_sm / (ms_best * 1e-3);       // per second per SM
    if (which == 0) ticks_per_s = cyc_best / (ms_best * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(KDE_ERR_CUDA, std::string("probe: ") + cudaGetErrorString(e));
  out[0] = rates[0];
  out[1] = rates[1];
  out[2] = rates[2];
  out[3] = sms;
  out[4] = ticks_per_s;
  return KDE_OK;
}
