// probe.cu -- measured FP64 FMA rate of the device, the denominator of the
// FP64-pipe rooflines (the secular kernels and the FP64 GEMM are bound by it).
#include <cuda_runtime.h>

#include "eig_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;     // independent FMA chains per thread
constexpr int kProbeIters = 2048;   // trips; each trip does kProbeChains x 4 FMAs

__device__ double g_probe_sink;

// Independent chains x <- x * a + b with |a| < 1: no memory traffic in the
// loop, enough warps per SM to hide the FMA latency.  The sum is written only
// when it equals an impossible value, so the chains stay live.
__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(double a, double b) {
  double x[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) x[j] = 1e-3 * (threadIdx.x + j);
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < kProbeChains; ++j) x[j] = fma(x[j], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) s += x[j];
  if (s == -1.2345e300) g_probe_sink = s;
}

}  // namespace

extern "C" int eig_fp64_fma_rate(int32_t device, int32_t reps, double* gflops, void* stream) {
  if (!gflops || reps < 1 || device < 0) return EIG_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return EIG_ECUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return EIG_ECUDA;
  }
  int rc = EIG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0, occ = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dfma_probe_kernel, kProbeThreads, 0) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = EIG_ECUDA;
  } else {
    const int blocks = sms * (occ > 0 ? occ : 1);
    const double fmas = (double)blocks * kProbeThreads * kProbeIters * 4.0 * kProbeChains;
    double best = 0.0;
    dfma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(0.9999999, 1e-7);  // warm-up
    for (int r = 0; r < reps && rc == EIG_OK; ++r) {
      float ms = 0.f;
      if (cudaEventRecord(e0, s) != cudaSuccess) rc = EIG_ECUDA;
      dfma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(0.9999999, 1e-7);
      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = EIG_ECUDA;
      else if (ms > 0.f)
        best = fmax(best, 2.0 * fmas / (ms * 1e-3) / 1e9);
    }
    *gflops = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
