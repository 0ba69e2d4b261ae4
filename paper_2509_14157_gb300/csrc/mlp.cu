// Learned Davidson guess: a per-amplitude MLP (features -> guess importance
// and diagonal-preconditioner correction), with its own training and
// inference kernels.
//
// Network: nin -> width -> width -> nout, ReLU on the two hidden layers,
// FP32 parameters. Training (FP32): forward, mean-squared-error loss with
// per-sample, per-output weights, backward, Adam. Inference: the same
// network in BF16 on the tensor cores (mma.sync, FP32 accumulation).
//
// The paper has no learned component; this is the library's extension for
// the Davidson start. Converged roots never depend on it: the Davidson
// convergence test and its products are the same whatever the start.
#include "../../include/fnocc.h"
#include "common.hpp"
#include "mlp.hpp"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

namespace fnocc {

namespace {

constexpr int NT = 256;

inline unsigned nblocks(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

// C = op(A) op(B) (+ bias) with element (m,k) of op(A) at A[m*sam + k*sak]
// and (k,n) of op(B) at B[k*sbk + n*sbn]; C[m*ldc + n]. Epilogue: + bias[n];
// mask (if set) zeroes C where mask[m*ldc + n] <= 0; relu_out (if set) gets
// max(C, 0). Split reduction: CTA z covers k in [z*kchunk, (z+1)*kchunk) and
// writes its partial product to C + z*M*ldc (no epilogue; summed in order by
// k_sum_splits).
struct SgemmArgs {
  int M, N, K, kchunk;
  const float *A;
  long long sam, sak;
  const float *B;
  long long sbk, sbn;
  float *C;
  long long ldc;
  const float *bias;
  float *relu_out;
  const float *mask;
  int split;
};

__global__ void __launch_bounds__(NT) k_sgemm(const SgemmArgs p) {
  constexpr int TB = 64, BKS = 16;
  __shared__ float As[BKS][TB + 1];
  __shared__ float Bs[BKS][TB + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TB, n0 = blockIdx.x * TB;
  const int kb = blockIdx.z * p.kchunk, ke = min(p.K, kb + p.kchunk);
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += BKS) {
    __syncthreads();
    for (int idx = tid; idx < TB * BKS; idx += NT) {
      const int kk = idx % BKS, r = idx / BKS;
      const int m = m0 + r, k = k0 + kk;
      As[kk][r] = (m < p.M && k < ke) ? p.A[m * p.sam + k * p.sak] : 0.f;
      const int c = idx % TB, kk2 = idx / TB;
      const int n = n0 + c, k2 = k0 + kk2;
      Bs[kk2][c] = (n < p.N && k2 < ke) ? p.B[k2 * p.sbk + n * p.sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKS; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  float *C = p.split ? p.C + (long long)blockIdx.z * p.M * p.ldc : p.C;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= p.N) continue;
      const long long o = (long long)m * p.ldc + n;
      float z = acc[i][j];
      if (!p.split) {
        if (p.bias) z += p.bias[n];
        if (p.mask && p.mask[o] <= 0.f) z = 0.f;
        if (p.relu_out) p.relu_out[o] = fmaxf(z, 0.f);
      }
      C[o] = z;
    }
  }
}

// out[i] = sum_z part[z * len + i], z in order
__global__ void k_sum_splits(const float *part, int nz, long long len, float *out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.f;
  for (int z = 0; z < nz; ++z) s += part[z * len + i];
  out[i] = s;
}

// BF16 inference layer: Z = X W + b (X: rows x K row-major FP32, W: K x N
// row-major FP32), relu_out = max(Z, 0). mma.sync m16n8k16, FP32
// accumulation; tile 64 x 64, K tile 32, 8 warps as 2 x 4.
__global__ void __launch_bounds__(NT) k_dense_bf16(int M, int N, int K, const float *__restrict__ X,
                                                   const float *__restrict__ W, const float *__restrict__ bias,
                                                   float *__restrict__ Z, float *__restrict__ relu_out) {
  constexpr int TBM = 64, TBN = 64, TBK = 32, LDS = 40;
  __shared__ __align__(16) __nv_bfloat16 As[TBM][LDS];
  __shared__ __align__(16) __nv_bfloat16 Bs[TBN][LDS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, tg = lane & 3;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  float acc[2][2][4] = {};
  for (int k0 = 0; k0 < K; k0 += TBK) {
    __syncthreads();
    for (int idx = tid; idx < TBM * TBK; idx += NT) {
      const int kk = idx % TBK, r = idx / TBK;
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = __float2bfloat16_rn((m < M && k < K) ? X[(long long)m * K + k] : 0.f);
    }
    for (int idx = tid; idx < TBN * TBK; idx += NT) {
      const int c = idx % TBN, kk = idx / TBN;
      const int n = n0 + c, k = k0 + kk;
      Bs[c][kk] = __float2bfloat16_rn((n < N && k < K) ? W[(long long)k * N + n] : 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < TBK; ks += 16) {
      unsigned a[2][4], b[2][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r0 = wm * 32 + mt * 16 + g, c0 = ks + 2 * tg;
        a[mt][0] = *reinterpret_cast<const unsigned *>(&As[r0][c0]);
        a[mt][1] = *reinterpret_cast<const unsigned *>(&As[r0 + 8][c0]);
        a[mt][2] = *reinterpret_cast<const unsigned *>(&As[r0][c0 + 8]);
        a[mt][3] = *reinterpret_cast<const unsigned *>(&As[r0 + 8][c0 + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int n = wn * 16 + nt * 8 + g;
        b[nt][0] = *reinterpret_cast<const unsigned *>(&Bs[n][ks + 2 * tg]);
        b[nt][1] = *reinterpret_cast<const unsigned *>(&Bs[n][ks + 2 * tg + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
              : "r"(a[mt][0]), "r"(a[mt][1]), "r"(a[mt][2]), "r"(a[mt][3]), "r"(b[nt][0]), "r"(b[nt][1]));
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = m0 + wm * 32 + mt * 16 + g + (e >= 2 ? 8 : 0);
        const int n = n0 + wn * 16 + nt * 8 + 2 * tg + (e & 1);
        if (m >= M || n >= N) continue;
        const float z = acc[mt][nt][e] + bias[n];
        Z[(long long)m * N + n] = z;
        if (relu_out) relu_out[(long long)m * N + n] = fmaxf(z, 0.f);
      }
}

// dY = 2 w (Y - T) / n; per-block partial losses (summed in order on the host)
__global__ void k_mse_grad(long long cnt, const float *Y, const float *T, const float *Wt, float inv_n, float *dY,
                           float *loss_part) {
  __shared__ float red[NT];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < cnt) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * Wt[i] * d * inv_n;
    l = Wt[i] * d * d * inv_n;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

__global__ void k_adam(long long n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_gather_rows(const float *src, int width, const int *rows, int nrows, float *dst) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nrows * width) return;
  const long long r = i / width, c = i - r * width;
  dst[i] = src[(long long)rows[r] * width + c];
}

__global__ void k_fill_f(float *x, float v, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

void sgemm(cudaStream_t s, SgemmArgs a) {
  a.split = 0;
  a.kchunk = a.K > 0 ? a.K : 1;
  dim3 grid(nblocks(a.N, 64), nblocks(a.M, 64), 1);
  k_sgemm<<<grid, NT, 0, s>>>(a);
  FNOCC_CUDA(cudaGetLastError());
}

// C (M x N, ldc = N) = op(A) op(B) with the reduction split into ordered
// partial products (large K, small output: the weight gradients)
void sgemm_split(cudaStream_t s, SgemmArgs a, DevBuf &part) {
  const int nz = std::max(1, std::min(64, a.K / 1024));
  const int kc = (a.K + nz - 1) / nz;
  a.kchunk = kc;
  const int z = (a.K + kc - 1) / kc;
  const long long len = (long long)a.M * a.ldc;
  part.reserve(sizeof(float) * (size_t)len * z);
  float *out = a.C;
  a.C = part.as<float>();
  a.split = 1;
  a.bias = nullptr;
  a.relu_out = nullptr;
  a.mask = nullptr;
  dim3 grid(nblocks(a.N, 64), nblocks(a.M, 64), z);
  k_sgemm<<<grid, NT, 0, s>>>(a);
  FNOCC_CUDA(cudaGetLastError());
  k_sum_splits<<<nblocks(len, 256), 256, 0, s>>>(part.as<float>(), z, len, out);
  FNOCC_CUDA(cudaGetLastError());
}

// counter-based generator (SplitMix64)
uint64_t splitmix64(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// x0 orbital-energy difference D = sum_p f_pp - sum_h f_hh; x1 spin-averaged
// two-body shift of the element's determinant (Epstein-Nesbet): over hole
// pairs and particle pairs +w_pq, over hole-particle pairs -w_pq, with w_pq =
// J_PP for two spin orbitals of one spatial orbital P and J_PQ - K_PQ / 2
// otherwise (the pair's <pq||pq> averaged over the spin of q); x2 highest
// hole energy; x3 lowest particle energy; x4 mean particle energy; x5 sum over
// particles of log10 of their virtual's natural occupation; x6 component
// (0, 1, 2); x7 variant (0..4). Every feature depends on spatial orbitals
// only, so a preconditioner built from them treats all spin couplings of a
// spatial configuration alike. g: antisymmetrised <pq||rs> of the n active
// spin orbitals (alpha even), occupied first.
__global__ void k_eom_features(int nh, int np, int o, int n, const int *htab, long long nhtup, const int *ptab,
                               long long nptup, const double *fdiag, const double *g, const float *vocc_log,
                               int comp, int variant, float *out) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nhtup * nptup) return;
  const long long hi = r / nptup, pi = r - hi * nptup;
  int idx[8];
  for (int k = 0; k < nh; ++k) idx[k] = htab[hi * nh + k];
  for (int k = 0; k < np; ++k) idx[nh + k] = o + ptab[pi * np + k];
  double sh = 0, sp = 0, hmax = 0, pmin = 0, occ = 0, en = 0;
  for (int k = 0; k < nh; ++k) {
    const double e = fdiag[idx[k]];
    sh += e;
    hmax = k == 0 ? e : fmax(hmax, e);
  }
  for (int k = 0; k < np; ++k) {
    const double e = fdiag[idx[nh + k]];
    sp += e;
    pmin = k == 0 ? e : fmin(pmin, e);
    occ += vocc_log ? vocc_log[idx[nh + k] - o] : 0.0;
  }
  const long long nn = n;
  for (int a = 0; a < nh + np; ++a)
    for (int b = a + 1; b < nh + np; ++b) {
      const long long p = idx[a], q = idx[b];
      double gv = g[((p * nn + q) * nn + p) * nn + q];
      if ((p >> 1) != (q >> 1)) gv = 0.5 * (gv + g[((p * nn + (q ^ 1)) * nn + p) * nn + (q ^ 1)]);
      en += ((a < nh) == (b < nh)) ? gv : -gv;
    }
  float *x = out + r * kMlpFeatures;
  x[0] = (float)(sp - sh);
  x[1] = (float)en;
  x[2] = (float)hmax;
  x[3] = (float)pmin;
  x[4] = np ? (float)(sp / np) : 0.f;
  x[5] = (float)occ;
  x[6] = (float)comp;
  x[7] = (float)variant;
}

__global__ void k_add_correction(long long n, const float *y, int stride, int col, double clamp, double *dg) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  dg[i] += fmin(clamp, fmax(-clamp, (double)y[i * stride + col]));
}

}  // namespace

void eom_features(cudaStream_t s, int nh, int np, int o, int n, const int *htab, long long nhtup, const int *ptab,
                  long long nptup, const double *fdiag, const double *g, const float *vocc_log, int comp, int variant,
                  float *out) {
  const long long cnt = nhtup * nptup;
  if (cnt <= 0) return;
  if (nh + np > 8) throw std::runtime_error("eom_features: more than 8 indices");
  k_eom_features<<<nblocks(cnt, 256), 256, 0, s>>>(nh, np, o, n, htab, nhtup, ptab, nptup, fdiag, g, vocc_log, comp,
                                                   variant, out);
  FNOCC_CUDA(cudaGetLastError());
}

void add_diag_correction(cudaStream_t s, long long n, const float *y, int stride, int col, double clamp, double *dg) {
  if (n <= 0) return;
  k_add_correction<<<nblocks(n, 256), 256, 0, s>>>(n, y, stride, col, clamp, dg);
  FNOCC_CUDA(cudaGetLastError());
}

Mlp::Mlp(int device, int nin, int width, int nout, uint64_t seed)
    : device_(device), nin_(nin), width_(width), nout_(nout) {
  FNOCC_CUDA(cudaSetDevice(device));
  FNOCC_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
  const int fan[3] = {nin, width, width}, outs[3] = {width, width, nout};
  size_t off = 0;
  for (int l = 0; l < 3; ++l) {
    woff_[l] = off;
    off += (size_t)fan[l] * outs[l];
    boff_[l] = off;
    off += outs[l];
  }
  nparam_ = off;
  // He-uniform weights from the counter-based generator, zero biases
  std::vector<float> h(nparam_, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < 3; ++l) {
    const float lim = std::sqrt(6.f / float(fan[l]));
    for (size_t i = 0; i < (size_t)fan[l] * outs[l]; ++i) {
      const double u = double(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
      h[woff_[l] + i] = float((2.0 * u - 1.0) * lim);
    }
  }
  params_.reserve(sizeof(float) * nparam_);
  adam_m_.reserve(sizeof(float) * nparam_);
  adam_v_.reserve(sizeof(float) * nparam_);
  grad_.reserve(sizeof(float) * nparam_);
  set_params(h.data());
  reset_optimizer();
}

Mlp::~Mlp() {
  if (stream_) cudaStreamDestroy(stream_);
}

void Mlp::set_params(const float *host) {
  FNOCC_CUDA(cudaSetDevice(device_));
  copy_after(params_.p, host, sizeof(float) * nparam_, cudaMemcpyHostToDevice, stream_);
}

void Mlp::get_params(float *host) const {
  FNOCC_CUDA(cudaSetDevice(device_));
  copy_after(host, params_.p, sizeof(float) * nparam_, cudaMemcpyDeviceToHost, stream_);
}

void Mlp::reset_optimizer() {
  FNOCC_CUDA(cudaMemsetAsync(adam_m_.p, 0, sizeof(float) * nparam_, stream_));
  FNOCC_CUDA(cudaMemsetAsync(adam_v_.p, 0, sizeof(float) * nparam_, stream_));
  adam_t_ = 0;
  FNOCC_CUDA(cudaStreamSynchronize(stream_));
}

const float *Mlp::W(int l) const { return params_.as<float>() + woff_[l]; }
const float *Mlp::b(int l) const { return params_.as<float>() + boff_[l]; }

// FP32 forward of n device rows keeping pre-activations and activations for
// the backward pass: [z1 | a1 | z2 | a2 | y]
void Mlp::forward_train(const float *X, int n) {
  act_.reserve(sizeof(float) * ((size_t)n * 4 * width_ + (size_t)n * nout_));
  float *z1 = act_.as<float>(), *a1 = z1 + (size_t)n * width_, *z2 = a1 + (size_t)n * width_,
        *a2 = z2 + (size_t)n * width_, *y = a2 + (size_t)n * width_;
  const int din[3] = {nin_, width_, width_}, dout[3] = {width_, width_, nout_};
  const float *in[3] = {X, a1, a2};
  float *zs[3] = {z1, z2, y}, *as[3] = {a1, a2, nullptr};
  for (int l = 0; l < 3; ++l) {
    SgemmArgs a{};
    a.M = n;
    a.N = dout[l];
    a.K = din[l];
    a.A = in[l];
    a.sam = din[l];
    a.sak = 1;
    a.B = W(l);
    a.sbk = dout[l];
    a.sbn = 1;
    a.C = zs[l];
    a.ldc = dout[l];
    a.bias = b(l);
    a.relu_out = as[l];
    sgemm(stream_, a);
  }
}

double Mlp::loss_grad(const float *X, const float *T, const float *Wt, int n) {
  FNOCC_CUDA(cudaSetDevice(device_));
  forward_train(X, n);
  float *z1 = act_.as<float>(), *a1 = z1 + (size_t)n * width_, *z2 = a1 + (size_t)n * width_,
        *a2 = z2 + (size_t)n * width_, *y = a2 + (size_t)n * width_;
  const long long cnt = (long long)n * nout_;
  dact_.reserve(sizeof(float) * ((size_t)cnt + 2 * (size_t)n * width_));
  float *dy = dact_.as<float>(), *d2 = dy + cnt, *d1 = d2 + (size_t)n * width_;
  const unsigned nb = nblocks(cnt, NT);
  lossp_.reserve(sizeof(float) * nb);
  k_mse_grad<<<nb, NT, 0, stream_>>>(cnt, y, T, Wt, 1.f / float(n), dy, lossp_.as<float>());
  FNOCC_CUDA(cudaGetLastError());
  ones_.reserve(sizeof(float));
  k_fill_f<<<1, 32, 0, stream_>>>(ones_.as<float>(), 1.f, 1);
  FNOCC_CUDA(cudaGetLastError());
  float *g = grad_.as<float>();
  const int din[3] = {nin_, width_, width_}, dout[3] = {width_, width_, nout_};
  const float *ain[3] = {X, a1, a2};
  float *dz[3] = {d1, d2, dy};
  const float *zpre[3] = {nullptr, z1, z2};  // pre-activation below layer l
  for (int l = 2; l >= 0; --l) {
    // dW_l = a_in^T dz_l (reduction over the rows), db_l = 1^T dz_l
    SgemmArgs a{};
    a.M = din[l];
    a.N = dout[l];
    a.K = n;
    a.A = ain[l];
    a.sam = 1;
    a.sak = din[l];
    a.B = dz[l];
    a.sbk = dout[l];
    a.sbn = 1;
    a.C = g + woff_[l];
    a.ldc = dout[l];
    sgemm_split(stream_, a, part_);
    SgemmArgs bb{};
    bb.M = 1;
    bb.N = dout[l];
    bb.K = n;
    bb.A = ones_.as<float>();
    bb.sam = 0;
    bb.sak = 0;
    bb.B = dz[l];
    bb.sbk = dout[l];
    bb.sbn = 1;
    bb.C = g + boff_[l];
    bb.ldc = dout[l];
    sgemm_split(stream_, bb, part_);
    if (l == 0) break;
    // dz_{l-1} = (dz_l W_l^T) * [z_{l-1} > 0]
    SgemmArgs c{};
    c.M = n;
    c.N = din[l];
    c.K = dout[l];
    c.A = dz[l];
    c.sam = dout[l];
    c.sak = 1;
    c.B = W(l);
    c.sbk = 1;
    c.sbn = dout[l];
    c.C = dz[l - 1];
    c.ldc = din[l];
    c.mask = zpre[l];
    sgemm(stream_, c);
  }
  std::vector<float> lp(nb);
  FNOCC_CUDA(cudaMemcpyAsync(lp.data(), lossp_.p, sizeof(float) * nb, cudaMemcpyDeviceToHost, stream_));
  FNOCC_CUDA(cudaStreamSynchronize(stream_));
  double loss = 0;
  for (float x : lp) loss += x;
  return loss;
}

void Mlp::adam_step(float lr, float b1, float b2, float eps) {
  ++adam_t_;
  const float c1 = 1.f - std::pow(b1, (float)adam_t_), c2 = 1.f - std::pow(b2, (float)adam_t_);
  k_adam<<<nblocks((long long)nparam_, NT), NT, 0, stream_>>>((long long)nparam_, params_.as<float>(),
                                                              grad_.as<float>(), adam_m_.as<float>(),
                                                              adam_v_.as<float>(), lr, b1, b2, c1, c2, eps);
  FNOCC_CUDA(cudaGetLastError());
}

void Mlp::train(const float *X, const float *T, const float *Wt, long long n, int epochs, int batch, float lr,
                uint64_t seed, double *history) {
  FNOCC_CUDA(cudaSetDevice(device_));
  data_.reserve(sizeof(float) * (size_t)n * (nin_ + 2 * nout_));
  float *dx = data_.as<float>(), *dt = dx + (size_t)n * nin_, *dw = dt + (size_t)n * nout_;
  FNOCC_CUDA(cudaMemcpyAsync(dx, X, sizeof(float) * n * nin_, cudaMemcpyHostToDevice, stream_));
  FNOCC_CUDA(cudaMemcpyAsync(dt, T, sizeof(float) * n * nout_, cudaMemcpyHostToDevice, stream_));
  FNOCC_CUDA(cudaMemcpyAsync(dw, Wt, sizeof(float) * n * nout_, cudaMemcpyHostToDevice, stream_));
  batch = (int)std::max<long long>(1, std::min<long long>(batch, n));
  mb_.reserve(sizeof(float) * (size_t)batch * (nin_ + 2 * nout_));
  rows_.reserve(sizeof(int) * batch);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  uint64_t st = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (long long i = n - 1; i > 0; --i) std::swap(order[i], order[splitmix64(st) % (uint64_t)(i + 1)]);
    double tot = 0;
    long long seen = 0;
    for (long long s = 0; s < n; s += batch) {
      const int nb = (int)std::min<long long>(batch, n - s);
      // (a copy from pageable memory is staged before the call returns)
      FNOCC_CUDA(cudaMemcpyAsync(rows_.p, order.data() + s, sizeof(int) * nb, cudaMemcpyHostToDevice, stream_));
      float *bx = mb_.as<float>(), *bt = bx + (size_t)batch * nin_, *bw = bt + (size_t)batch * nout_;
      k_gather_rows<<<nblocks((long long)nb * nin_, NT), NT, 0, stream_>>>(dx, nin_, rows_.as<int>(), nb, bx);
      k_gather_rows<<<nblocks((long long)nb * nout_, NT), NT, 0, stream_>>>(dt, nout_, rows_.as<int>(), nb, bt);
      k_gather_rows<<<nblocks((long long)nb * nout_, NT), NT, 0, stream_>>>(dw, nout_, rows_.as<int>(), nb, bw);
      FNOCC_CUDA(cudaGetLastError());
      tot += loss_grad(bx, bt, bw, nb) * nb;
      seen += nb;
      adam_step(lr, 0.9f, 0.999f, 1e-8f);
    }
    if (history) history[ep] = tot / double(std::max<long long>(1, seen));
  }
  FNOCC_CUDA(cudaStreamSynchronize(stream_));
}

// BF16 inference of n device rows on `stream`, in row chunks so that the
// hidden activations stay small
void Mlp::infer_bf16(const float *X, long long n, float *Y, cudaStream_t stream, DevBuf &scratch) const {
  FNOCC_CUDA(cudaSetDevice(device_));
  const long long chunk = 1 << 18;
  scratch.reserve(sizeof(float) * (size_t)std::min<long long>(n, chunk) * 4 * width_);
  for (long long r0 = 0; r0 < n; r0 += chunk) {
    const int m = (int)std::min<long long>(chunk, n - r0);
    float *z1 = scratch.as<float>(), *a1 = z1 + (size_t)m * width_, *z2 = a1 + (size_t)m * width_,
          *a2 = z2 + (size_t)m * width_;
    dim3 g1(nblocks(width_, 64), nblocks(m, 64));
    k_dense_bf16<<<g1, NT, 0, stream>>>(m, width_, nin_, X + r0 * nin_, W(0), b(0), z1, a1);
    k_dense_bf16<<<g1, NT, 0, stream>>>(m, width_, width_, a1, W(1), b(1), z2, a2);
    dim3 g3(nblocks(nout_, 64), nblocks(m, 64));
    k_dense_bf16<<<g3, NT, 0, stream>>>(m, nout_, width_, a2, W(2), b(2), Y + r0 * nout_, nullptr);
    FNOCC_CUDA(cudaGetLastError());
  }
}

// FP32 inference (the training path's forward)
void Mlp::infer_fp32(const float *X, long long n, float *Y) {
  FNOCC_CUDA(cudaSetDevice(device_));
  forward_train(X, (int)n);
  const float *y = act_.as<float>() + (size_t)n * 4 * width_;
  FNOCC_CUDA(cudaMemcpyAsync(Y, y, sizeof(float) * n * nout_, cudaMemcpyDeviceToDevice, stream_));
  FNOCC_CUDA(cudaStreamSynchronize(stream_));
}

}  // namespace fnocc

// ---- C ABI ------------------------------------------------------------------------

namespace {

template <class F>
fnocc_status mlp_guarded(fnocc_mlp *m, F &&fn) {
  try {
    return fn();
  } catch (const fnocc::CudaError &e) {
    if (m) m->err = e.what();
    return FNOCC_E_CUDA;
  } catch (const std::bad_alloc &e) {
    if (m) m->err = e.what();
    return FNOCC_E_NOMEM;
  } catch (const std::exception &e) {
    if (m) m->err = e.what();
    return FNOCC_E_INVALID;
  }
}

// parameter file: 8-byte tag, then int32 version, nin, width, nout, int64
// parameter count, then the FP32 parameters (host byte order, the layout of
// fnocc_mlp_get_params)
constexpr char kMlpTag[8] = {'F', 'N', 'O', 'C', 'C', 'M', 'L', 'P'};
constexpr int32_t kMlpVersion = 1;

struct MlpFileHeader {
  char tag[8];
  int32_t version, nin, width, nout;
  int64_t nparam;
};

}  // namespace

extern "C" {

fnocc_status fnocc_mlp_create(fnocc_mlp **out, int device, int nin, int width, int nout, unsigned long long seed) {
  if (!out || nin != fnocc::kMlpFeatures || width < 1 || width > 4096 || nout != fnocc::kMlpOutputs)
    return FNOCC_E_INVALID;
  *out = nullptr;
  auto *m = new (std::nothrow) fnocc_mlp;
  if (!m) return FNOCC_E_NOMEM;
  fnocc_status st = mlp_guarded(m, [&]() -> fnocc_status {
    m->net.reset(new fnocc::Mlp(device, nin, width, nout, seed));
    return FNOCC_OK;
  });
  if (st != FNOCC_OK) {
    delete m;
    return st;
  }
  *out = m;
  return FNOCC_OK;
}

void fnocc_mlp_destroy(fnocc_mlp *m) { delete m; }

const char *fnocc_mlp_last_error(const fnocc_mlp *m) { return m ? m->err.c_str() : "null network"; }

size_t fnocc_mlp_param_count(const fnocc_mlp *m) { return m && m->net ? m->net->nparam() : 0; }

fnocc_status fnocc_mlp_get_params(fnocc_mlp *m, float *params, size_t len) {
  if (!m || !params || len != m->net->nparam()) return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    m->net->get_params(params);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_mlp_set_params(fnocc_mlp *m, const float *params, size_t len) {
  if (!m || !params || len != m->net->nparam()) return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    m->net->set_params(params);
    m->net->reset_optimizer();
    return FNOCC_OK;
  });
}

fnocc_status fnocc_mlp_forward(fnocc_mlp *m, const float *x, long long n, float *y, int bf16) {
  if (!m || !x || !y || n <= 0 || (!bf16 && n > (1LL << 24))) return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    fnocc::Mlp &net = *m->net;
    FNOCC_CUDA(cudaSetDevice(net.device()));
    fnocc::DevBuf dx, dy, scratch;
    dx.reserve(sizeof(float) * n * net.nin());
    dy.reserve(sizeof(float) * n * net.nout());
    FNOCC_CUDA(cudaMemcpyAsync(dx.p, x, sizeof(float) * n * net.nin(), cudaMemcpyHostToDevice, net.stream()));
    if (bf16)
      net.infer_bf16(dx.as<float>(), n, dy.as<float>(), net.stream(), scratch);
    else
      net.infer_fp32(dx.as<float>(), n, dy.as<float>());
    FNOCC_CUDA(cudaMemcpyAsync(y, dy.p, sizeof(float) * n * net.nout(), cudaMemcpyDeviceToHost, net.stream()));
    FNOCC_CUDA(cudaStreamSynchronize(net.stream()));
    return FNOCC_OK;
  });
}

fnocc_status fnocc_mlp_loss_grad(fnocc_mlp *m, const float *x, const float *t, const float *w, long long n,
                                 double *loss, float *grad) {
  if (!m || !x || !t || !w || n <= 0 || n > (1LL << 24)) return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    fnocc::Mlp &net = *m->net;
    FNOCC_CUDA(cudaSetDevice(net.device()));
    fnocc::DevBuf d;
    const size_t nx = (size_t)n * net.nin(), ny = (size_t)n * net.nout();
    d.reserve(sizeof(float) * (nx + 2 * ny));
    float *dx = d.as<float>(), *dt = dx + nx, *dw = dt + ny;
    FNOCC_CUDA(cudaMemcpyAsync(dx, x, sizeof(float) * nx, cudaMemcpyHostToDevice, net.stream()));
    FNOCC_CUDA(cudaMemcpyAsync(dt, t, sizeof(float) * ny, cudaMemcpyHostToDevice, net.stream()));
    FNOCC_CUDA(cudaMemcpyAsync(dw, w, sizeof(float) * ny, cudaMemcpyHostToDevice, net.stream()));
    const double l = net.loss_grad(dx, dt, dw, (int)n);
    if (loss) *loss = l;
    if (grad) fnocc::copy_after(grad, net.grad(), sizeof(float) * net.nparam(), cudaMemcpyDeviceToHost, net.stream());
    return FNOCC_OK;
  });
}

fnocc_status fnocc_mlp_train(fnocc_mlp *m, const float *x, const float *t, const float *w, long long n, int epochs,
                             int batch, float lr, unsigned long long seed, double *history) {
  if (!m || !x || !t || !w || n <= 0 || n > (1LL << 31) - 1 || epochs < 0 || batch <= 0 || !(lr > 0))
    return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    m->net->train(x, t, w, n, epochs, batch, lr, seed, history);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_mlp_save(fnocc_mlp *m, const char *path) {
  if (!m || !path) return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    const fnocc::Mlp &net = *m->net;
    std::vector<float> p(net.nparam());
    net.get_params(p.data());
    MlpFileHeader hd{};
    std::memcpy(hd.tag, kMlpTag, sizeof(hd.tag));
    hd.version = kMlpVersion;
    hd.nin = net.nin();
    hd.width = net.width();
    hd.nout = net.nout();
    hd.nparam = (int64_t)p.size();
    FILE *f = std::fopen(path, "wb");
    if (!f) throw std::runtime_error(std::string("cannot open ") + path + " for writing");
    const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    if (std::fclose(f) != 0 || !ok) throw std::runtime_error(std::string("cannot write ") + path);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_mlp_load(fnocc_mlp *m, const char *path) {
  if (!m || !path) return FNOCC_E_INVALID;
  return mlp_guarded(m, [&]() -> fnocc_status {
    fnocc::Mlp &net = *m->net;
    FILE *f = std::fopen(path, "rb");
    if (!f) throw std::runtime_error(std::string("cannot open ") + path);
    MlpFileHeader hd{};
    std::vector<float> p(net.nparam());
    bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1;
    const bool match = ok && std::memcmp(hd.tag, kMlpTag, sizeof(hd.tag)) == 0 && hd.version == kMlpVersion &&
                       hd.nin == net.nin() && hd.width == net.width() && hd.nout == net.nout() &&
                       hd.nparam == (int64_t)p.size();
    ok = match && std::fread(p.data(), sizeof(float), p.size(), f) == p.size();
    std::fclose(f);
    if (!match)
      throw std::runtime_error(std::string(path) + ": not a parameter file of this network's shape");
    if (!ok) throw std::runtime_error(std::string(path) + ": truncated");
    net.set_params(p.data());
    net.reset_optimizer();
    return FNOCC_OK;
  });
}

}  // extern "C"
