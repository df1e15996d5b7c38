// fd_peak.cu -- fd_measure_fp64_peak: the FP64 throughput this GPU sustains on
// independent fused multiply-adds, the denominator of the FP64 kernels'
// roofline (they are bound by the FP64 pipe, not by memory).
#include <cuda_runtime.h>

#include <cstdio>

#include "fd_internal.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

__device__ double g_sink;

// Every thread runs kChains independent chains x <- x * b + c for `iters`
// steps: 2 kChains iters flops per thread, no memory traffic in the loop. The
// sum is stored only if it equals `never` (the caller passes a value the chains
// cannot reach), so the compiler must keep the arithmetic.
__global__ void __launch_bounds__(128) dfma_probe_kernel(double b, double c, int iters,
                                                         double never) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == never) g_sink = s;
}

}  // namespace

extern "C" fd_status fd_measure_fp64_peak(int32_t device, int32_t iters, double *tflops,
                                          double *elapsed_ms) {
  if (!tflops || iters < 1) return fdk_fail(FD_ERR_INVALID_ARG, "fd_measure_fp64_peak: bad argument");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  cudaDeviceProp pr{};
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&pr, device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaSetDevice(prev);
    return fdk_fail(FD_ERR_CUDA, "fd_measure_fp64_peak: no usable device");
  }
  // four 128-thread blocks per SM: four warps per sub-partition, enough to keep
  // the FP64 pipe issuing with eight independent chains each
  const int blocks = pr.multiProcessorCount * 4;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    // the multiplier keeps |x| bounded: x -> x b + c with b < 1 converges to c / (1 - b)
    dfma_probe_kernel<<<blocks, 128, 0, s>>>(0.999999, 1e-6, iters / 8 + 1, -1.0);  // warm-up
    cudaEventRecord(e0, s);
    dfma_probe_kernel<<<blocks, 128, 0, s>>>(0.999999, 1e-6, iters, -1.0);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof msg, "fd_measure_fp64_peak: %s", cudaGetErrorString(e));
    return fdk_fail(FD_ERR_CUDA, msg);
  }
  const double flops = 2.0 * kChains * static_cast<double>(iters) * blocks * 128.0;
  *tflops = flops / (static_cast<double>(ms) * 1e-3) / 1e12;
  if (elapsed_ms) *elapsed_ms = ms;
  return FD_OK;
}
