// FMA throughput microbenchmark: the measured FP64 and FP32 peaks the benchmark reports the
// pair kernels against.  The paper has no counterpart; this is a measurement aid.
//
// Every thread runs eight independent chains a <- fma(a, b, c) (b slightly below 1, so each chain
// converges to c / (1 - b) and stays finite), enough independent work per warp to keep the FMA
// pipe busy at full occupancy.  The grid is the occupancy limit times the SM count.  One call
// times a launch sized to take about the requested time with CUDA events, after a calibration
// launch, and returns the best of three: flops = 2 x 8 x iterations x threads.
#include <cuda_runtime.h>

#include <algorithm>

#include "sph2d_internal.h"

namespace sph2d {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T b, T c, T* __restrict__ out) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(0.25) + T(j) * T(0.01) + T(threadIdx.x) * T(1e-6);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[tid] = s;                                    // keeps every chain live
}

template <typename T>
static sph2d_status measure(int device, double seconds, double* tflops) {
  if (cudaSetDevice(device) != cudaSuccess) return SPH2D_ERR_CUDA;
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<T>, 256, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = std::max(1, per_sm) * std::max(1, sms);
  const int64_t threads = int64_t(blocks) * 256;
  T* out = nullptr;
  if (cudaMalloc(&out, size_t(threads) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return SPH2D_ERR_OUT_OF_MEMORY;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T b = T(1) - T(1.0 / 1048576.0), c = T(1e-3);
  auto run = [&](int iters) -> float {
    cudaEventRecord(e0);
    fma_peak_kernel<T><<<blocks, 256>>>(iters, b, c, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  int iters = 16;
  float ms = run(iters);                           // warm-up and calibration
  while (ms < 5.0f && iters < (1 << 26)) {
    iters *= 4;
    ms = run(iters);
  }
  iters = int(std::min(double(1 << 28), std::max(1.0, iters * (seconds * 1e3 / std::max(ms, 1e-3f)))));
  double best = 1e30;
  for (int r = 0; r < 3; ++r) best = std::min(best, double(run(iters)));
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return SPH2D_ERR_CUDA;
  const double flops = 2.0 * 8.0 * 16.0 * double(iters) * double(threads);
  *tflops = flops / (best * 1e-3) / 1e12;
  return SPH2D_OK;
}

}  // namespace sph2d

extern "C" sph2d_status sph2d_measure_fma_peak(int device, int precision, double seconds, double* tflops) {
  if (!tflops || !(seconds > 0.0) || seconds > 10.0 || (precision != 0 && precision != 1))
    return SPH2D_ERR_INVALID_ARG;
  return precision == 0 ? sph2d::measure<double>(device, seconds, tflops)
                        : sph2d::measure<float>(device, seconds, tflops);
}
