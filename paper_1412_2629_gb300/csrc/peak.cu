// FP32 CUDA-core peak of the current device, measured: the denominator of the Schwarz
// kernel's roofline (that kernel is bound by FP32 arithmetic, not by memory).
//
// Every thread runs eight independent chains of fused multiply-adds x <- a x + b, so the
// FMA pipes stay busy with no memory traffic; a, b are run-time values (no folding) with
// |a| < 1, so the chains stay finite.  One FFMA is 2 flop.
#include "dd.h"
#include "dd_kernels.hpp"

namespace dd {

constexpr int PEAK_CHAINS = 8, PEAK_UNROLL = 16, PEAK_THREADS = 512;

__global__ void __launch_bounds__(PEAK_THREADS) ffma_peak_kernel(float* out, int iters, float a, float b) {
  float x[PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) s += x[i];
  if (s == -1.0f) out[0] = s;   // never true for these inputs; keeps the chains live
}

// The same with FP64 chains (the FP64 operator of the reliable update is bound by GB300's FP64
// rate).  Fewer iterations: the FP64 units are a small fraction of the FP32 ones.
__global__ void __launch_bounds__(PEAK_THREADS) dfma_peak_kernel(double* out, int iters, double a, double b) {
  double x[PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = 1e-3 * (double)threadIdx.x + (double)i;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < PEAK_CHAINS; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < PEAK_CHAINS; ++i) s += x[i];
  if (s == -1.0) out[0] = s;   // never true for these inputs; keeps the chains live
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_fp64_peak(int duration_ms, double* burst_tflops, double* sustained_tflops) {
  if (duration_ms < 1 || !burst_tflops || !sustained_tflops) return DD_ERR_INVALID;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_peak_kernel, PEAK_THREADS, 0);
  if (sms <= 0 || per_sm <= 0) return DD_ERR_CUDA;
  const int grid = sms * per_sm, iters = 64;
  const double flop = 2.0 * grid * PEAK_THREADS * (double)iters * PEAK_UNROLL * PEAK_CHAINS;
  double* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dd_status rc = DD_OK;
  if (cudaMalloc(&out, 16) != cudaSuccess) return DD_ERR_OOM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = DD_ERR_CUDA;
  double best = 0.0, total_ms = 0.0, total_flop = 0.0;
  for (int rep = 0; rc == DD_OK && (rep < 3 || total_ms < duration_ms); ++rep) {
    cudaEventRecord(e0, st);
    dfma_peak_kernel<<<grid, PEAK_THREADS, 0, st>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) { rc = DD_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0) continue;   // first launch: warm-up
    best = fmax(best, flop / (ms * 1e-3) / 1e12);
    total_ms += ms;
    total_flop += flop;
  }
  if (rc == DD_OK) {
    *burst_tflops = best;
    *sustained_tflops = total_flop / (total_ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}

extern "C" dd_status dd_fp32_peak(int duration_ms, double* burst_tflops, double* sustained_tflops) {
  if (duration_ms < 1 || !burst_tflops || !sustained_tflops) return DD_ERR_INVALID;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ffma_peak_kernel, PEAK_THREADS, 0);
  if (sms <= 0 || per_sm <= 0) return DD_ERR_CUDA;
  const int grid = sms * per_sm, iters = 4096;
  const double flop = 2.0 * grid * PEAK_THREADS * (double)iters * PEAK_UNROLL * PEAK_CHAINS;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dd_status rc = DD_OK;
  if (cudaMalloc(&out, 16) != cudaSuccess) return DD_ERR_OOM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = DD_ERR_CUDA;
  double best = 0.0, total_ms = 0.0, total_flop = 0.0;
  for (int rep = 0; rc == DD_OK && (rep < 3 || total_ms < duration_ms); ++rep) {
    cudaEventRecord(e0, st);
    ffma_peak_kernel<<<grid, PEAK_THREADS, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) { rc = DD_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0) continue;   // first launch: warm-up
    best = fmax(best, flop / (ms * 1e-3) / 1e12);
    total_ms += ms;
    total_flop += flop;
  }
  if (rc == DD_OK) {
    *burst_tflops = best;
    *sustained_tflops = total_flop / (total_ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}
