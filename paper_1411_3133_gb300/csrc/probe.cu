// Measured arithmetic peak of this GPU (lb_fma_peak): the denominator of the
// ALU roofline of the FP64 step, which is bound by the FP64 units rather than
// by HBM.
//
// Every thread runs eight independent fused multiply-add chains
// a <- a * m + c (m slightly below 1, so the chains converge instead of
// overflowing), four rounds per loop trip; 2 flops per FMA. The grid holds eight
// 256-thread blocks per SM, enough warps to hide the FMA latency. The
// result is stored only when it equals an impossible value, which keeps the
// chains alive without a memory stream.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbgm.h"
#include "launch.h"

namespace lbgm {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ inline float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ inline double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T m, T c, T* sink) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {  // 4 x kChains FMAs per loop trip
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma_t(a[k], m, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1.2345e30)) sink[0] = s;
}

lb_status probe_fail(lb_status s, const std::string& m) {
  set_last_error_noctx(m);
  return s;
}

template <typename T>
lb_status run_probe(cudaStream_t st, double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return probe_fail(LB_ERR_CUDA, "lb_fma_peak: no CUDA device");
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return probe_fail(LB_ERR_CUDA, "lb_fma_peak: cudaMalloc failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 8 * sms;
  const double threads = double(blocks) * kThreads;
  const T m = T(0.999999), c = T(1e-6);
  double best = 0.0;
  lb_status status = LB_OK;
  // warm-up; the lengthening runs below warm up further
  cudaEventRecord(e0, st);
  k_fma_probe<T><<<blocks, kThreads, 0, st>>>(256, m, c, sink);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  int iters = 1 << 10;
  int timed = 0;
  while (timed < 5) {
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, kThreads, 0, st>>>(iters, m, c, sink);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      status = probe_fail(LB_ERR_CUDA, "lb_fma_peak: probe launch failed");
      break;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
      status = probe_fail(LB_ERR_CUDA, "lb_fma_peak: event timing failed");
      break;
    }
    if (ms < 50.f && iters < (1 << 24)) {  // too short to time: lengthen
      iters *= 2;
      continue;
    }
    const double f = 2.0 * 4 * kChains * double(iters) * threads / (ms * 1e-3);
    if (f > best) best = f;
    ++timed;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (status == LB_OK) *flops_per_s = best;
  return status;
}

}  // namespace
}  // namespace lbgm

using namespace lbgm;

extern "C" lb_status lb_fma_peak(lb_precision precision, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s) return probe_fail(LB_ERR_ARG, "lb_fma_peak: flops_per_s is NULL");
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (precision == LB_FP64) return run_probe<double>(st, flops_per_s);
  if (precision == LB_FP32) return run_probe<float>(st, flops_per_s);
  return probe_fail(LB_ERR_ARG, "lb_fma_peak: precision must be LB_FP64 or LB_FP32");
}
