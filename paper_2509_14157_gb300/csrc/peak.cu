// FP64 throughput probe of the device: the denominators of the FP64
// roofline fractions (the contraction kernels of the FP64 path issue FP64
// FMAs; the tensor-core FP64 form, mma.sync m8n8k4, is measured beside it).
//
// Both kernels run long chains of independent multiply-adds from registers
// (no memory traffic in the loop) on every SM and are timed with CUDA events;
// the best of several launches is reported in TFLOP/s (2 flops per
// multiply-add).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/fnocc.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp64_fma(double b, double c, int iters, double *sink) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = threadIdx.x * 1e-9 + j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1.2345e300) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true: keeps the chains live
}

// one warp-wide m8n8k4 FP64 product per call: D (8x8) += A (8x4) * B (4x8)
__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kThreads) k_fp64_dmma(double a, double b, int iters, double *sink) {
  double d[kChains][2];
#pragma unroll
  for (int j = 0; j < kChains; ++j) d[j][0] = d[j][1] = threadIdx.x * 1e-9 + j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) dmma(d[j][0], d[j][1], a, b);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += d[j][0] + d[j][1];
  if (s == 1.2345e300) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" fnocc_status fnocc_fp64_peak(int device, double *fma_tflops, double *dmma_tflops) {
  if (!fma_tflops || !dmma_tflops) return FNOCC_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FNOCC_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return FNOCC_E_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    return FNOCC_E_CUDA;
  fnocc_status st = FNOCC_OK;
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  const int blocks = sms * 8;  // 8 resident CTAs of 256 threads per SM
  const int iters = 1 << 14;
  double best_fma = 0, best_dmma = 0;
  if (cudaMalloc(&sink, sizeof(double) * blocks * kThreads) != cudaSuccess) return FNOCC_E_NOMEM;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = FNOCC_E_CUDA;
  } else {
    for (int rep = 0; rep < 6 && st == FNOCC_OK; ++rep) {
      float ms = 0;
      cudaEventRecord(e0, s);
      k_fp64_fma<<<blocks, kThreads, 0, s>>>(1.0000001, 1e-7, iters, sink);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0) {
        st = FNOCC_E_CUDA;
        break;
      }
      const double flops = 2.0 * kChains * double(iters) * blocks * kThreads;
      if (rep > 0) best_fma = std::max(best_fma, flops / (ms * 1e-3) / 1e12);
      cudaEventRecord(e0, s);
      k_fp64_dmma<<<blocks, kThreads, 0, s>>>(1.0000001, 1e-7, iters / 4, sink);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0) {
        st = FNOCC_E_CUDA;
        break;
      }
      // per warp and call: 8 x 8 x 4 multiply-adds
      const double dflops = 2.0 * 256.0 * kChains * double(iters / 4) * blocks * (kThreads / 32);
      if (rep > 0) best_dmma = std::max(best_dmma, dflops / (ms * 1e-3) / 1e12);
    }
    if (st == FNOCC_OK && cudaGetLastError() != cudaSuccess) st = FNOCC_E_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(sink);
  *fma_tflops = best_fma;
  *dmma_tflops = best_dmma;
  return st;
}
