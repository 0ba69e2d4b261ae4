// Allocation-free Davidson projection, for callers that cannot allocate
// device memory themselves: a process whose device memory belongs to another
// allocator (a framework's caching allocator or a pool sized up front) must
// not call cudaMalloc/cudaFree behind that allocator's back, and a
// latency-sensitive caller avoids cudaFree because it synchronises the whole
// device.
//
// Same result as fnocc_multi_dot, but the partial sums of the two-pass
// reduction live in a fixed file-scope device array instead of
// context-owned memory. The array is 256 x 64 doubles (128 KiB) and is
// reserved on every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fnocc.h"

namespace {

constexpr int kBlocks = 256;   // blocks of the first pass
constexpr int kMaxVec = 64;    // largest nvec the fixed scratch holds
constexpr int kMaxDevices = 64;

// Scratch of the partial sums: [nvec][kBlocks]. Pass 1 writes every element
// pass 2 reads, so nothing needs clearing between calls; the array keeps the
// last call's partial sums.
static __device__ __align__(256) double g_partials[kMaxVec * kBlocks];

double *g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__global__ void k_noalloc_dot_partial(long long n, const double *x, const double *Y, long long ld, double *part) {
  __shared__ double red[256];
  const int j = blockIdx.y;
  const double *y = Y + j * ld;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[j * kBlocks + blockIdx.x] = red[0];
}

__global__ void k_noalloc_dot_final(int nblk, int nvec, const double *part, double *dots) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[j * kBlocks + b];
  dots[j] = s;
}

}  // namespace

extern "C" fnocc_status fnocc_multi_dot_noalloc(const double *x, const double *Y, size_t n, size_t ld, int nvec,
                                                double *dots, void *stream) {
  if (!x || !Y || !dots || n == 0 || ld < n) return FNOCC_E_INVALID;
  if (nvec < 1 || nvec > kMaxVec) return FNOCC_E_INVALID;  // beyond the fixed scratch
  // an error left pending by the caller's own work stays theirs to read: do
  // not launch, and do not clear it, so the checks below see only this call
  if (cudaPeekAtLastError() != cudaSuccess) return FNOCC_E_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FNOCC_E_CUDA;
  double *part = nullptr;
  {
    // once per device, with that device current: the device address of the
    // scratch (its host-side name is only a stand-in for it)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return FNOCC_E_CUDA;
      g_partials_addr[dev] = static_cast<double *>(p);
    }
    part = g_partials_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long blocks = ((long long)n + 256 * 8 - 1) / (256 * 8);
  const int nblk = (int)(blocks < 1 ? 1 : (blocks > kBlocks ? kBlocks : blocks));
  dim3 grid(nblk, nvec);
  k_noalloc_dot_partial<<<grid, 256, 0, s>>>((long long)n, x, Y, (long long)ld, part);
  if (cudaGetLastError() != cudaSuccess) return FNOCC_E_CUDA;
  k_noalloc_dot_final<<<(nvec + 127) / 128, 128, 0, s>>>(nblk, nvec, part, dots);
  if (cudaGetLastError() != cudaSuccess) return FNOCC_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FNOCC_E_CUDA;
  return FNOCC_OK;
}
