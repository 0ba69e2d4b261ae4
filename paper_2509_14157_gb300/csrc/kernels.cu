// CUDA kernels of libfnocc (sm_103a). FP64 throughout.
//
// The contraction kernel is a gather-GEMM-scatter: every operand element is
// addressed through per-dimension offset tables (DMap), so index permutations,
// block slices of the integral tensors and antisymmetry-packed index tuples
// (i<j<k, a<b, ...) are read and written in place without materialised
// transposes. On this part FP64 FMA issue (about two FP64 FMAs per clock per
// SM) is the bound of every contraction, so the kernel is a register-tiled
// SIMT FP64 GEMM: a 64x64 tile per 256-thread block, 4x4 outputs per thread,
// K staged through shared memory 16 at a time.
#include "common.hpp"

#include <cuda_bf16.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <mutex>

namespace fnocc {

namespace {

constexpr int BK = 16, NT = 256;

struct GemmParams {
  long long M, N, K;
  long long kchunk;
  double alpha;
  const double *A;
  const double *B;
  double *C;
  DMap arow, acol, brow, bcol, crow, ccol;
  long long tiles_n;
  int atomic;
  int accumulate;
};

__device__ __forceinline__ long long map_off(const DMap &mp, long long m) {
  long long off = 0;
  for (int g = mp.ng - 1; g >= 0; --g) {
    long long q = m / mp.n[g];
    long long r = m - q * mp.n[g];
    off += mp.tab[g][r];
    m = q;
  }
  return off;
}

// Tiled FP64 gather-GEMM. 256 threads as 16 x 16, each computing a TM x TN
// micro-tile, so a block covers 16*TM rows and 16*TN columns; K is
// staged through shared memory 16 at a time. PART: write the block's partial
// product of one K chunk (grid.y) to part[z][m * N + n] for an ordered
// split-K reduction instead of updating C.
template <int TM, int TN, bool PART>
__global__ void __launch_bounds__(NT) k_gather_gemm(const GemmParams p, double *part) {
  constexpr int TBM = 16 * TM, TBN = 16 * TN;
  __shared__ double As[BK][TBM];
  __shared__ double Bs[BK][TBN];
  __shared__ long long arow_s[TBM], crow_s[TBM], bcol_s[TBN], ccol_s[TBN], acol_s[BK], brow_s[BK];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long tile = blockIdx.x;
  const long long m0 = (tile / p.tiles_n) * TBM;
  const long long n0 = (tile % p.tiles_n) * TBN;
  const long long kb = (long long)blockIdx.y * p.kchunk;
  const long long ke = min(p.K, kb + p.kchunk);
  if (tid < TBM) {
    long long m = m0 + tid;
    arow_s[tid] = m < p.M ? map_off(p.arow, m) : 0;
    if (!PART) crow_s[tid] = m < p.M ? map_off(p.crow, m) : 0;
  } else if (tid < TBM + TBN) {
    long long n = n0 + tid - TBM;
    bcol_s[tid - TBM] = n < p.N ? map_off(p.bcol, n) : 0;
    if (!PART) ccol_s[tid - TBM] = n < p.N ? map_off(p.ccol, n) : 0;
  }
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (long long k0 = kb; k0 < ke; k0 += BK) {
    __syncthreads();
    if (tid < BK) {
      long long k = k0 + tid;
      acol_s[tid] = k < ke ? map_off(p.acol, k) : 0;
    } else if (tid < 2 * BK) {
      long long k = k0 + tid - BK;
      brow_s[tid - BK] = k < ke ? map_off(p.brow, k) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TM; ++r) {  // TBM * BK / NT = TM elements per thread
      int idx = tid + NT * r;
      int kk = idx % BK, row = idx / BK;
      bool ok = (m0 + row < p.M) && (k0 + kk < ke);
      As[kk][row] = ok ? p.A[arow_s[row] + acol_s[kk]] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < TN; ++r) {
      int idx = tid + NT * r;
      int col = idx % TBN, kk = idx / TBN;
      bool ok = (n0 + col < p.N) && (k0 + kk < ke);
      Bs[kk][col] = ok ? p.B[brow_s[kk] + bcol_s[col]] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  double *dst_part = PART ? part + (long long)blockIdx.y * p.M * p.N : nullptr;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    long long m = m0 + ty * TM + i;
    if (m >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      long long n = n0 + tx * TN + j;
      if (n >= p.N) continue;
      if (PART) {
        dst_part[m * p.N + n] = acc[i][j];
      } else {
        double *dst = p.C + crow_s[ty * TM + i] + ccol_s[tx * TN + j];
        double val = p.alpha * acc[i][j];
        if (p.accumulate)
          *dst += val;
        else
          *dst = val;
      }
    }
  }
}

// BF16 three-slice split GEMM on the tensor cores (mixed precision). Each
// gathered FP64 operand element is rounded to FP32 and split exactly into
// three BF16 slices x = x0 + x1 + x2 (8 significant bits each, 24 in all);
// the six slice products with i + j <= 2 are accumulated in FP32 by
// mma.sync m16n8k16 (the products themselves are exact). Block tile 64 x 64,
// K tile 32, 8 warps as 2 x 4, each warp 32 x 16 outputs (2 x 2 MMA tiles).
// Relative error about 1e-7 of the summed magnitudes; the solvers finish in
// FP64.
template <bool PART>
__global__ void __launch_bounds__(NT) k_gather_gemm_bf16x3(const GemmParams p, double *part) {
  constexpr int TBM = 64, TBN = 64, TBK = 32, LDS = 40;  // padded row stride (bf16) avoids bank conflicts
  __shared__ __align__(16) __nv_bfloat16 As[3][TBM][LDS];
  __shared__ __align__(16) __nv_bfloat16 Bs[3][TBN][LDS];
  __shared__ long long arow_s[TBM], crow_s[TBM], bcol_s[TBN], ccol_s[TBN], acol_s[TBK], brow_s[TBK];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;
  const int g = lane >> 2, tg = lane & 3;
  const long long tile = blockIdx.x;
  const long long m0 = (tile / p.tiles_n) * TBM;
  const long long n0 = (tile % p.tiles_n) * TBN;
  const long long kb = (long long)blockIdx.y * p.kchunk;
  const long long ke = min(p.K, kb + p.kchunk);
  if (tid < TBM) {
    long long m = m0 + tid;
    arow_s[tid] = m < p.M ? map_off(p.arow, m) : 0;
    crow_s[tid] = (!PART && m < p.M) ? map_off(p.crow, m) : 0;
  } else if (tid < TBM + TBN) {
    long long n = n0 + tid - TBM;
    bcol_s[tid - TBM] = n < p.N ? map_off(p.bcol, n) : 0;
    ccol_s[tid - TBM] = (!PART && n < p.N) ? map_off(p.ccol, n) : 0;
  }
  float acc[2][2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  for (long long k0 = kb; k0 < ke; k0 += TBK) {
    __syncthreads();
    if (tid < TBK) {
      long long k = k0 + tid;
      acol_s[tid] = k < ke ? map_off(p.acol, k) : 0;
    } else if (tid < 2 * TBK) {
      long long k = k0 + tid - TBK;
      brow_s[tid - TBK] = k < ke ? map_off(p.brow, k) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < (TBM * TBK) / NT; ++r) {
      int idx = tid + NT * r;
      int kk = idx % TBK, row = idx / TBK;
      bool ok = (m0 + row < p.M) && (k0 + kk < ke);
      float xf = ok ? (float)p.A[arow_s[row] + acol_s[kk]] : 0.f;
      __nv_bfloat16 h = __float2bfloat16_rn(xf);
      float r1 = xf - __bfloat162float(h);
      __nv_bfloat16 md = __float2bfloat16_rn(r1);
      float r2 = r1 - __bfloat162float(md);
      As[0][row][kk] = h;
      As[1][row][kk] = md;
      As[2][row][kk] = __float2bfloat16_rn(r2);
    }
#pragma unroll
    for (int r = 0; r < (TBN * TBK) / NT; ++r) {
      int idx = tid + NT * r;
      int col = idx % TBN, kk = idx / TBN;
      bool ok = (n0 + col < p.N) && (k0 + kk < ke);
      float xf = ok ? (float)p.B[brow_s[kk] + bcol_s[col]] : 0.f;
      __nv_bfloat16 h = __float2bfloat16_rn(xf);
      float r1 = xf - __bfloat162float(h);
      __nv_bfloat16 md = __float2bfloat16_rn(r1);
      float r2 = r1 - __bfloat162float(md);
      Bs[0][col][kk] = h;
      Bs[1][col][kk] = md;
      Bs[2][col][kk] = __float2bfloat16_rn(r2);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < TBK; ks += 16) {
      unsigned a[3][2][4], b[3][2][2];
#pragma unroll
      for (int s = 0; s < 3; ++s) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int r0 = wm * 32 + mt * 16 + g;
          const int c0 = ks + 2 * tg;
          a[s][mt][0] = *reinterpret_cast<const unsigned *>(&As[s][r0][c0]);
          a[s][mt][1] = *reinterpret_cast<const unsigned *>(&As[s][r0 + 8][c0]);
          a[s][mt][2] = *reinterpret_cast<const unsigned *>(&As[s][r0][c0 + 8]);
          a[s][mt][3] = *reinterpret_cast<const unsigned *>(&As[s][r0 + 8][c0 + 8]);
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int n = wn * 16 + nt * 8 + g;
          b[s][nt][0] = *reinterpret_cast<const unsigned *>(&Bs[s][n][ks + 2 * tg]);
          b[s][nt][1] = *reinterpret_cast<const unsigned *>(&Bs[s][n][ks + 2 * tg + 8]);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3 - i; ++j)
#pragma unroll
          for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
              asm volatile(
                  "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                  "{%0,%1,%2,%3};\n"
                  : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
                  : "r"(a[i][mt][0]), "r"(a[i][mt][1]), "r"(a[i][mt][2]), "r"(a[i][mt][3]), "r"(b[j][nt][0]),
                    "r"(b[j][nt][1]));
    }
  }
  double *dst_part = PART ? part + (long long)blockIdx.y * p.M * p.N : nullptr;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int rl = wm * 32 + mt * 16 + g + (e >= 2 ? 8 : 0);
        const int cl = wn * 16 + nt * 8 + 2 * tg + (e & 1);
        const long long m = m0 + rl, n = n0 + cl;
        if (m >= p.M || n >= p.N) continue;
        if (PART) {
          dst_part[m * p.N + n] = (double)acc[mt][nt][e];
        } else {
          double *dst = p.C + crow_s[rl] + ccol_s[cl];
          double val = p.alpha * (double)acc[mt][nt][e];
          if (p.accumulate)
            *dst += val;
          else
            *dst = val;
        }
      }
}

// Small outputs (M*N <= 256): blocks split K; inside a block the K chunk is
// staged 256 offsets at a time, warp w owns outputs w, w + 8, ... (at most
// 32), its lanes stride over K and a shuffle reduction closes each output.
// Partials go to part[blockIdx.x][M*N]; every useful multiply-add is done once.
__global__ void __launch_bounds__(256) k_gemm_small(const GemmParams p, double *part) {
  __shared__ long long acol_s[256], brow_s[256], ar_s[256], bc_s[256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const long long O = p.M * p.N;
  if (t < O) {
    ar_s[t] = map_off(p.arow, t / p.N);
    bc_s[t] = map_off(p.bcol, t % p.N);
  }
  const long long kb = (long long)blockIdx.x * p.kchunk;
  const long long ke = min(p.K, kb + p.kchunk);
  double acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.0;
  for (long long k0 = kb; k0 < ke; k0 += 256) {
    __syncthreads();
    long long k = k0 + t;
    acol_s[t] = k < ke ? map_off(p.acol, k) : 0;
    brow_s[t] = k < ke ? map_off(p.brow, k) : 0;
    __syncthreads();
    const int nk = (int)min((long long)256, ke - k0);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int o = warp + 8 * j;
      if (o < O) {
        const long long ab = ar_s[o], bb = bc_s[o];
        double s = acc[j];
        for (int kk = lane; kk < nk; kk += 32) s = fma(p.A[ab + acol_s[kk]], p.B[brow_s[kk] + bb], s);
        acc[j] = s;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int o = warp + 8 * j;
    if (o < O) {  // uniform across the warp
      double v = acc[j];
      for (int w = 16; w > 0; w >>= 1) v += __shfl_down_sync(0xffffffffu, v, w);
      if (lane == 0) part[(long long)blockIdx.x * O + o] = v;
    }
  }
}

// C[crow(m) + ccol(n)] (+)= alpha * sum_z part[z][m * N + n], z in order
__global__ void k_reduce_partials(const GemmParams p, const double *part, int nz) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long O = p.M * p.N;
  if (idx >= O) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += part[(long long)z * O + idx];
  double *dst = p.C + map_off(p.crow, idx / p.N) + map_off(p.ccol, idx % p.N);
  *dst = p.accumulate ? *dst + p.alpha * s : p.alpha * s;
}

// GEMV (N = 1): one thread per row, the K loop in registers, x offsets staged
// in shared memory. Used for the Davidson linear combinations and Fock builds.
__global__ void __launch_bounds__(256) k_gemv_rows(const GemmParams p) {
  __shared__ long long acol_s[256], brow_s[256];
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ar = m < p.M ? map_off(p.arow, m) : 0;
  const long long bc = map_off(p.bcol, 0);
  double acc = 0.0;
  for (long long k0 = 0; k0 < p.K; k0 += 256) {
    __syncthreads();
    long long k = k0 + threadIdx.x;
    acol_s[threadIdx.x] = k < p.K ? map_off(p.acol, k) : 0;
    brow_s[threadIdx.x] = k < p.K ? map_off(p.brow, k) : 0;
    __syncthreads();
    const int nk = (int)min((long long)256, p.K - k0);
    if (m < p.M)
      for (int kk = 0; kk < nk; ++kk) acc = fma(p.A[ar + acol_s[kk]], p.B[brow_s[kk] + bc], acc);
  }
  if (m < p.M) {
    double *dst = p.C + map_off(p.crow, m) + map_off(p.ccol, 0);
    *dst = p.accumulate ? *dst + p.alpha * acc : p.alpha * acc;
  }
}

__global__ void k_gather_axpy(long long M, double alpha, const double *A, DMap arow, double *C, DMap crow) {
  long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= M) return;
  C[map_off(crow, m)] += alpha * A[map_off(arow, m)];
}

// permutation tables for up to 4 elements, generated on the device side once
__constant__ signed char c_perm[5][24][4];
__constant__ signed char c_psign[5][24];
__constant__ int c_pcount[5];

__device__ __forceinline__ void dense_strides(int nh, int np, int o, int v, long long *sh, long long *sp) {
  long long s = 1;
  for (int k = np - 1; k >= 0; --k) { sp[k] = s; s *= v; }
  for (int k = nh - 1; k >= 0; --k) { sh[k] = s; s *= o; }
}

// Dense work tensors (the contraction engine's operands and accumulators)
// hold each index of a space in the canonical order of the engine's tuple
// tables: beta spin orbitals (odd p) first, then alpha, ascending within
// each, so that the elements of one spin block are contiguous. Position of
// spin orbital x in a space of n (even) spin orbitals, and its inverse.
__device__ __forceinline__ int canon_pos(int x, int n) { return (x & 1) ? (x >> 1) : (n >> 1) + (x >> 1); }
__device__ __forceinline__ int canon_index(int d, int n) { return d < (n >> 1) ? 2 * d + 1 : 2 * (d - (n >> 1)); }

// canonical: Y in the canonical order above (the engine's accumulators),
// else in spin-orbital order
__global__ void k_antisym_pack(const double *Y, int nh, int np, int o, int v, const int *htab, long long nhtup,
                               const int *ptab, long long nptup, double *out, double scale, int accumulate,
                               int canonical) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nhtup * nptup) return;
  long long hi = r / nptup, pi = r - hi * nptup;
  long long sh[4], sp[4];
  dense_strides(nh, np, o, v, sh, sp);
  int h[4], pv[4];
  for (int k = 0; k < nh; ++k) h[k] = canonical ? canon_pos(htab[hi * nh + k], o) : htab[hi * nh + k];
  for (int k = 0; k < np; ++k) pv[k] = canonical ? canon_pos(ptab[pi * np + k], v) : ptab[pi * np + k];
  double acc = 0.0;
  const int nph = c_pcount[nh], npp = c_pcount[np];
  for (int a = 0; a < nph; ++a) {
    long long offh = 0;
    for (int k = 0; k < nh; ++k) offh += sh[k] * h[c_perm[nh][a][k]];
    double part = 0.0;
    for (int b = 0; b < npp; ++b) {
      long long off = offh;
      for (int k = 0; k < np; ++k) off += sp[k] * pv[c_perm[np][b][k]];
      part += c_psign[np][b] * Y[off];
    }
    acc += c_psign[nh][a] * part;
  }
  acc *= scale;
  out[r] = accumulate ? out[r] + acc : acc;
}

// dense in the canonical order (an engine operand)
__global__ void k_unpack_dense(const double *packed, int nh, int np, int o, int v, const int *htab, long long nhtup,
                               const int *ptab, long long nptup, double *dense) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nhtup * nptup) return;
  long long hi = r / nptup, pi = r - hi * nptup;
  long long sh[4], sp[4];
  dense_strides(nh, np, o, v, sh, sp);
  int h[4], pv[4];
  for (int k = 0; k < nh; ++k) h[k] = canon_pos(htab[hi * nh + k], o);
  for (int k = 0; k < np; ++k) pv[k] = canon_pos(ptab[pi * np + k], v);
  const double val = packed[r];
  const int nph = c_pcount[nh], npp = c_pcount[np];
  for (int a = 0; a < nph; ++a) {
    long long offh = 0;
    for (int k = 0; k < nh; ++k) offh += sh[k] * h[c_perm[nh][a][k]];
    for (int b = 0; b < npp; ++b) {
      long long off = offh;
      for (int k = 0; k < np; ++k) off += sp[k] * pv[c_perm[np][b][k]];
      dense[off] = c_psign[nh][a] * c_psign[np][b] * val;
    }
  }
}

// insertion sort of a short index list; flips sgn per swap, sets dup on a
// repeated index
__device__ __forceinline__ void sort_small(int *t, int n, int &sgn, bool &dup) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && t[j - 1] >= t[j]; --j) {
      if (t[j - 1] == t[j]) dup = true;
      const int x = t[j - 1];
      t[j - 1] = t[j];
      t[j] = x;
      sgn = -sgn;
    }
}

// Dense antisymmetric tensor [o^NH v^NP] (canonical index order, see
// canon_pos) from its packed unique elements, as a coalesced gather (every
// dense element written once, no prior clear):
// block b owns the outer indices (holes and all but the last NI particles),
// its threads stride over the inner NI particle indices, which are the
// fastest-varying part of the dense layout. dense = sign(sorting
// permutation) * packed[rank], 0 on repeated indices. hr / pr: rank prefix
// tables of the hole / particle tuple lists (TupleTable::rank), staged in
// shared memory (v <= 160).
template <int NH, int NP>
__global__ void __launch_bounds__(256) k_unpack_blocks(const double *__restrict__ packed, int o, int v,
                                                       const long long *__restrict__ hr,
                                                       const long long *__restrict__ pr, long long nptup,
                                                       long long inner, double *__restrict__ dense) {
  constexpr int NI = NP < 3 ? NP : 3, NO = NP - NI;
  __shared__ long long prs[NP * 161];
  for (int i = threadIdx.x; i < NP * (v + 1); i += blockDim.x) prs[i] = pr[i];
  const long long outer = blockIdx.x;
  long long rem = outer;
  int po[NO > 0 ? NO : 1], hh[NH > 0 ? NH : 1];
#pragma unroll
  for (int k = NO - 1; k >= 0; --k) {
    po[k] = canon_index((int)(rem % v), v);
    rem /= v;
  }
#pragma unroll
  for (int k = NH - 1; k >= 0; --k) {
    hh[k] = canon_index((int)(rem % o), o);
    rem /= o;
  }
  int sgn0 = 1;
  bool dup0 = false;
  sort_small(hh, NH, sgn0, dup0);
  long long hrank = 0;
#pragma unroll
  for (int i = 0; i < NH; ++i) hrank += hr[i * (o + 1) + hh[i]] - hr[i * (o + 1) + (i ? hh[i - 1] + 1 : 0)];
  __syncthreads();
  if (dup0) {
    for (long long j = threadIdx.x; j < inner; j += blockDim.x) dense[outer * inner + j] = 0.0;
    return;
  }
  const double *pk = packed + hrank * nptup;
  double *dst = dense + outer * inner;
  const unsigned uv = (unsigned)v;
  for (long long j = threadIdx.x; j < inner; j += blockDim.x) {
    int q[NP];
#pragma unroll
    for (int k = 0; k < NO; ++k) q[k] = po[k];
    unsigned r = (unsigned)j;
#pragma unroll
    for (int k = NP - 1; k >= NO; --k) {
      q[k] = canon_index((int)(r % uv), v);
      r /= uv;
    }
    int sgn = sgn0;
    bool dup = false;
#pragma unroll
    for (int i = 1; i < NP; ++i)
#pragma unroll
      for (int k = i; k > 0; --k)
        if (q[k - 1] >= q[k]) {
          if (q[k - 1] == q[k]) dup = true;
          const int x = q[k - 1];
          q[k - 1] = q[k];
          q[k] = x;
          sgn = -sgn;
        }
    double val = 0.0;
    if (!dup) {
      long long prank = 0;
#pragma unroll
      for (int i = 0; i < NP; ++i) prank += prs[i * (v + 1) + q[i]] - prs[i * (v + 1) + (i ? q[i - 1] + 1 : 0)];
      val = sgn * __ldg(pk + prank);
    }
    dst[j] = val;
  }
}

__global__ void k_fill(double *x, double val, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = val;
}

__global__ void k_axpby(long long n, double a, const double *x, double b, double *y) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_scale_mask(long long n, double *x, const unsigned char *mask) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && !mask[i]) x[i] = 0.0;
}

__global__ void k_jacobi_update(long long n, const double *r, const double *d, double *t) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) t[i] += r[i] / d[i];
}

__global__ void k_precondition(long long n, const double *r, const double *d, double theta,
                               const unsigned char *mask, double *out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double den = theta - d[i];
  if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
  out[i] = (!mask || mask[i]) ? r[i] / den : 0.0;
}

__global__ void k_gather_idx(long long n, const long long *idx, const double *src, double *dst) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_scatter_idx(long long n, const long long *idx, const double *src, double *dst) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = src[i];
}

// y[i] (+)= sum_j coef[j] * X[j * ld + i]: one streaming pass over the k
// rows (each row read coalesced), coefficients staged in shared memory
__global__ void k_lincomb(long long n, const double *__restrict__ X, long long ld, int k,
                          const double *__restrict__ coef, double *__restrict__ y, int accumulate) {
  extern __shared__ double cs[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = coef[j];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    double acc = accumulate ? y[i] : 0.0;
    const double *xp = X + i;
    for (int j = 0; j < k; ++j) acc = fma(cs[j], __ldg(xp + (long long)j * ld), acc);
    y[i] = acc;
  }
}

// partial dot products: grid (gx, nvec)
__global__ void k_dot_partial(long long n, const double *x, const double *Y, long long ld, double *part) {
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
  if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_dot_final(int gx, int nvec, const double *part, double *dots) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < gx; ++b) s += part[j * gx + b];
  dots[j] = s;
}

__global__ void k_absmax_partial(long long n, const double *x, double *part) {
  __shared__ double rm[256], rs[256];
  double m = 0.0, s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double a = x[i];
    m = fmax(m, fabs(a));
    s = fma(a, a, s);
    if (a != a) m = CUDART_INF;  // NaN marks as infinite
  }
  rm[threadIdx.x] = m;
  rs[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rm[threadIdx.x] = fmax(rm[threadIdx.x], rm[threadIdx.x + w]);
      rs[threadIdx.x] += rs[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rm[0];
    part[2 * blockIdx.x + 1] = rs[0];
  }
}

__global__ void k_absmax_final(int gx, const double *part, double *out) {
  if (threadIdx.x != 0) return;
  double m = 0.0, s = 0.0;
  for (int b = 0; b < gx; ++b) {
    m = fmax(m, part[2 * b]);
    s += part[2 * b + 1];
  }
  out[0] = m;
  out[1] = s;
}

// <PQ||RS> over spin orbitals P = 2p + s from spatial (pq|rs)
__global__ void k_spin_eri(const double *e, int n, double *g) {
  const long long ns = 2LL * n;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= ns * ns * ns * ns) return;
  long long S = idx % ns, R = (idx / ns) % ns, Q = (idx / (ns * ns)) % ns, P = idx / (ns * ns * ns);
  int p = P >> 1, q = Q >> 1, r = R >> 1, s = S >> 1;
  int sp = P & 1, sq = Q & 1, sr = R & 1, ss = S & 1;
  double val = 0.0;
  const long long n2 = (long long)n * n;
  if (sp == sr && sq == ss) val += e[(p * (long long)n + r) * n2 + q * (long long)n + s];
  if (sp == ss && sq == sr) val -= e[(p * (long long)n + s) * n2 + q * (long long)n + r];
  g[idx] = val;
}

__global__ void k_spin_h(const double *h, int n, double *hso) {
  const int ns = 2 * n;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ns * ns) return;
  int P = idx / ns, Q = idx % ns;
  hso[idx] = ((P & 1) == (Q & 1)) ? h[(P >> 1) * n + (Q >> 1)] : 0.0;
}

__global__ void k_normal_order(const double *h, const double *g, int n, int o, double *f) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int p = idx / n, q = idx % n;
  const long long n3 = (long long)n * n * n, n2 = (long long)n * n;
  double s = h[idx];
  for (int i = 0; i < o; ++i) s += g[p * n3 + i * n2 + q * (long long)n + i];
  f[idx] = s;
}

__global__ void k_eref(const double *h, const double *g, int n, int o, double *out) {
  __shared__ double r1[256], r2[256];
  const long long n3 = (long long)n * n * n, n2 = (long long)n * n;
  double a = 0.0, b = 0.0;
  for (int idx = threadIdx.x; idx < o * o; idx += blockDim.x) {
    int i = idx / o, j = idx % o;
    if (i == j) a += h[i * n + i];
    b += g[i * n3 + j * n2 + i * (long long)n + j];
  }
  r1[threadIdx.x] = a;
  r2[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = r1[0];
    out[1] = 0.5 * r2[0];
  }
}

__global__ void k_t1_mats(const double *t1, int o, int v, double *Lm, double *Mm) {
  const int n = o + v;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int p = idx / n, q = idx % n;
  double l = (p == q) ? 1.0 : 0.0, m = l;
  if (p < o && q >= o) l = -t1[p * v + (q - o)];  // L[i, a] = -t_i^a
  if (p >= o && q < o) m = t1[q * v + (p - o)];   // M[a, i] = t_i^a
  Lm[idx] = l;
  Mm[idx] = m;
}

// One-block cyclic Jacobi for symmetric A (n <= 128), tournament ordering.
__global__ void k_jacobi_eig(double *Ag, int n, double *evals, double *V, int *info) {
  extern __shared__ double A[];
  __shared__ double cs[64], sn[64];
  __shared__ int pp[64], qq[64];
  __shared__ double red[512], red2[512];
  __shared__ int stop;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) {
    A[idx] = Ag[idx];
    V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  }
  const int npad = n + (n & 1);
  const int half = npad / 2;
  int sweep;
  __syncthreads();
  for (sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < n * n; idx += nt) {
      double a = A[idx];
      tot += a * a;
      if (idx / n != idx % n) off += a * a;
    }
    red[tid] = off;
    red2[tid] = tot;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) {
        red[tid] += red[tid + w];
        red2[tid] += red2[tid + w];
      }
      __syncthreads();
    }
    if (tid == 0) stop = (red[0] <= 1e-30 * red2[0] || red[0] < 1e-300) ? 1 : 0;
    __syncthreads();
    if (stop) break;
    for (int rnd = 0; rnd < npad - 1; ++rnd) {
      if (tid < half) {
        int k = tid;
        int a = (k == 0) ? 0 : ((k - 1 + rnd) % (npad - 1)) + 1;
        int kb = npad - 1 - k;
        int b = ((kb - 1 + rnd) % (npad - 1)) + 1;
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[p * n + q];
          if (fabs(apq) > 1e-300) {
            double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = q < n ? q : -1;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nt) {  // rows
        int k = idx / n, j = idx % n;
        int p = pp[k], q = qq[k];
        if (q < 0) continue;
        double c = cs[k], s = sn[k];
        double apj = A[p * n + j], aqj = A[q * n + j];
        A[p * n + j] = c * apj - s * aqj;
        A[q * n + j] = s * apj + c * aqj;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nt) {  // columns and V
        int k = idx / n, i = idx % n;
        int p = pp[k], q = qq[k];
        if (q < 0) continue;
        double c = cs[k], s = sn[k];
        double aip = A[i * n + p], aiq = A[i * n + q];
        A[i * n + p] = c * aip - s * aiq;
        A[i * n + q] = s * aip + c * aiq;
        double vip = V[i * n + p], viq = V[i * n + q];
        V[i * n + p] = c * vip - s * viq;
        V[i * n + q] = s * vip + c * viq;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += nt) evals[i] = A[i * n + i];
  if (tid == 0) info[0] = sweep;
}

__global__ void k_permute_columns(const double *in, int rows, int cols_in, const int *perm, int cols_out, double *out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols_out) return;
  int i = idx / cols_out, j = idx % cols_out;
  out[idx] = in[i * cols_in + perm[j]];
}

__global__ void k_fix_phase(double *c, int rows, int cols) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  int best = 0;
  double bv = -1.0;
  for (int i = 0; i < rows; ++i) {
    double a = fabs(c[i * cols + j]);
    if (a > bv) { bv = a; best = i; }
  }
  if (c[best * cols + j] < 0)
    for (int i = 0; i < rows; ++i) c[i * cols + j] = -c[i * cols + j];
}

__global__ void k_lincomb3(long long n, double *out, const double *a, double alpha, const double *b, double beta,
                           const double *c) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + alpha * b[i] + beta * c[i];
}

__global__ void k_mp2(const double *g, const double *fd, int n, int o, double *t) {
  const int v = n - o;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)o * o * v * v) return;
  int b = idx % v, a = (idx / v) % v, j = (idx / (v * v)) % o, i = idx / ((long long)v * v * o);
  const long long n3 = (long long)n * n * n, n2 = (long long)n * n;
  double num = g[(o + a) * n3 + (o + b) * n2 + i * (long long)n + j];
  double den = fd[i] + fd[j] - fd[o + a] - fd[o + b];
  t[idx] = (i == j || a == b) ? 0.0 : num / den;
}

__global__ void k_diag(const double *a, int n, double *d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = a[i * n + i];
}

__global__ void k_alpha_block(const double *in, int nso, double *out) {
  int m = nso / 2;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  int p = idx / m, q = idx % m;
  out[idx] = in[(2 * p) * nso + 2 * q];
}

__global__ void k_eom_diag(const double *fd, int o, int nh, int np, const int *htab, long long nhtup, const int *ptab,
                           long long nptup, double *d) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nhtup * nptup) return;
  long long hi = r / nptup, pi = r - hi * nptup;
  double s = 0.0;
  for (int k = 0; k < np; ++k) s += fd[o + ptab[pi * np + k]];
  for (int k = 0; k < nh; ++k) s -= fd[htab[hi * nh + k]];
  d[r] = s;
}

__global__ void k_ms_mask(int nh, int np, const int *htab, long long nhtup, const int *ptab, long long nptup, int ms2,
                          unsigned char *mask) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nhtup * nptup) return;
  long long hi = r / nptup, pi = r - hi * nptup;
  int s = 0;
  for (int k = 0; k < np; ++k) s += (ptab[pi * np + k] & 1) ? -1 : 1;
  for (int k = 0; k < nh; ++k) s -= (htab[hi * nh + k] & 1) ? -1 : 1;
  mask[r] = (s == ms2) ? 1 : 0;
}

__global__ void k_cc_den(const double *fd, int o, int rank, const int *htab, long long nhtup, const int *ptab,
                         long long nptup, double *d) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nhtup * nptup) return;
  long long hi = r / nptup, pi = r - hi * nptup;
  double s = 0.0;
  for (int k = 0; k < rank; ++k) s += fd[htab[hi * rank + k]] - fd[o + ptab[pi * rank + k]];
  d[r] = s;
}

inline unsigned blocks_for(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

// The permutation tables live in constant memory, one copy per device: fill
// each device's copy once (thread-safe; contexts may run on host threads).
void ensure_perm_tables() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  FNOCC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) throw std::runtime_error("device index out of range");
  if (done[dev]) return;
  signed char perm[5][24][4] = {};
  signed char sgn[5][24] = {};
  int cnt[5] = {};
  for (int k = 0; k <= 4; ++k) {
    int a[4] = {0, 1, 2, 3};
    int c = 0;
    do {
      int inv = 0;
      for (int x = 0; x < k; ++x)
        for (int y = x + 1; y < k; ++y)
          if (a[x] > a[y]) ++inv;
      for (int x = 0; x < 4; ++x) perm[k][c][x] = (signed char)(x < k ? a[x] : 0);
      sgn[k][c] = (inv & 1) ? -1 : 1;
      ++c;
    } while (std::next_permutation(a, a + k));
    cnt[k] = c;
  }
  // complete before any stream can launch a reader (see copy_now)
  FNOCC_CUDA(cudaMemcpyToSymbolAsync(c_perm, perm, sizeof(perm), 0, cudaMemcpyHostToDevice, cudaStreamPerThread));
  FNOCC_CUDA(cudaMemcpyToSymbolAsync(c_psign, sgn, sizeof(sgn), 0, cudaMemcpyHostToDevice, cudaStreamPerThread));
  FNOCC_CUDA(cudaMemcpyToSymbolAsync(c_pcount, cnt, sizeof(cnt), 0, cudaMemcpyHostToDevice, cudaStreamPerThread));
  FNOCC_CUDA(cudaStreamSynchronize(cudaStreamPerThread));
  done[dev] = true;
}

inline void post(const Launch &L) {
  FNOCC_CUDA(cudaGetLastError());
  if (L.counter) ++*L.counter;
}

}  // namespace

int gather_gemm(const Launch &L, long long M, long long N, long long K, double alpha, const double *A,
                 const DMap &arow, const DMap &acol, const double *B, const DMap &brow, const DMap &bcol, double *C,
                 const DMap &crow, const DMap &ccol, bool accumulate, long long asize, long long bsize,
                 long long csize, int shape_req) {
  if (M <= 0 || N <= 0) return -1;
  if (arow.maxoff + acol.maxoff >= asize || brow.maxoff + bcol.maxoff >= bsize || crow.maxoff + ccol.maxoff >= csize ||
      arow.maxoff < 0 || acol.maxoff < 0 || brow.maxoff < 0 || bcol.maxoff < 0 || crow.maxoff < 0 || ccol.maxoff < 0)
    throw std::runtime_error("gather_gemm: index map exceeds operand bounds");
  GemmParams p;
  p.M = M;
  p.N = N;
  p.K = K > 0 ? K : 1;
  p.alpha = alpha;
  p.A = A;
  p.B = B;
  p.C = C;
  p.arow = arow;
  p.acol = acol;
  p.brow = brow;
  p.bcol = bcol;
  p.crow = crow;
  p.ccol = ccol;
  const bool mixed = L.precision == 1 && M >= 32 && N >= 32 && p.K >= 32;
  // tile shape with the least padding (ties: the square 64 x 64 tile)
  static const int shapes[kTileShapes][2] = {{4, 4}, {8, 2}, {2, 8}, {8, 1}, {1, 8}};
  int shape = 0;
  double best_pad = -1;
  for (int sidx = 0; sidx < kTileShapes; ++sidx) {
    long long bm = 16 * shapes[sidx][0], bn = 16 * shapes[sidx][1];
    double pad = double((M + bm - 1) / bm * bm) * double((N + bn - 1) / bn * bn);
    if (best_pad < 0 || pad < best_pad * 0.999) {
      best_pad = pad;
      shape = sidx;
    }
  }
  if (shape_req >= 0 && shape_req < kTileShapes) shape = shape_req;
  const long long tbm = mixed ? 64 : 16 * shapes[shape][0], tbn = mixed ? 64 : 16 * shapes[shape][1];
  p.tiles_n = (N + tbn - 1) / tbn;
  long long tiles = ((M + tbm - 1) / tbm) * p.tiles_n;
  p.accumulate = accumulate ? 1 : 0;
  auto launch_tiled = [&](dim3 grid, bool part_mode, double *partp) {
    if (mixed) {
      if (part_mode)
        k_gather_gemm_bf16x3<true><<<grid, NT, 0, L.stream>>>(p, partp);
      else
        k_gather_gemm_bf16x3<false><<<grid, NT, 0, L.stream>>>(p, partp);
      return;
    }
#define FNOCC_TILED(a, b)                                                                       \
  if (part_mode)                                                                               \
    k_gather_gemm<a, b, true><<<grid, NT, 0, L.stream>>>(p, partp);                            \
  else                                                                                         \
    k_gather_gemm<a, b, false><<<grid, NT, 0, L.stream>>>(p, partp);
    switch (shape) {
      case 0: FNOCC_TILED(4, 4) break;
      case 1: FNOCC_TILED(8, 2) break;
      case 2: FNOCC_TILED(2, 8) break;
      case 3: FNOCC_TILED(8, 1) break;
      default: FNOCC_TILED(1, 8) break;
    }
#undef FNOCC_TILED
  };
  GemmProfile *pr = (L.prof && L.prof->enabled) ? L.prof : nullptr;
  int e0 = -1;
  auto begin = [&]() {
    if (!pr) return;
    while (pr->pool.size() < 2 * pr->pairs.size() + 2) {
      cudaEvent_t ev;
      FNOCC_CUDA(cudaEventCreate(&ev));
      pr->pool.push_back(ev);
    }
    e0 = (int)(2 * pr->pairs.size());
    FNOCC_CUDA(cudaEventRecord(pr->pool[e0], L.stream));
  };
  auto end = [&](int path) {
    if (!pr) return;
    FNOCC_CUDA(cudaEventRecord(pr->pool[e0 + 1], L.stream));
    pr->pairs.push_back({e0, e0 + 1});
    pr->flops.push_back(2.0 * double(M) * double(N) * double(p.K));
    pr->path.push_back(path);
    if (pr->pairs.size() >= 4096) pr->fold();
  };
  p.atomic = 0;
  const long long want = 2 * (long long)L.sms;
  const long long O = M * N;
  // GEMV shape with enough rows: one thread per row
  if (N == 1 && M >= 2048) {
    p.kchunk = p.K;
    begin();
    k_gemv_rows<<<blocks_for(M, 256), 256, 0, L.stream>>>(p);
    post(L);
    end(3);
    return -1;
  }
  // tiny outputs: one thread per output, K split over blocks, ordered reduction
  if (O <= 256) {
    // FP64 issue is slow per SM: spread K over about two blocks per SM
    // (chunks of at least 64) so that the whole GPU works on the few outputs
    long long nblk = std::min<long long>(std::max<long long>(1, p.K / 64), 2 * (long long)L.sms);
    long long kchunk = (p.K + nblk - 1) / nblk;
    nblk = (p.K + kchunk - 1) / kchunk;
    p.kchunk = kchunk;
    if (!L.partials) throw std::runtime_error("gather_gemm: no partial-sum scratch");
    L.partials->reserve(sizeof(double) * (size_t)(nblk * O));
    begin();
    k_gemm_small<<<(unsigned)nblk, 256, 0, L.stream>>>(p, L.partials->d());
    post(L);
    k_reduce_partials<<<blocks_for(O, 256), 256, 0, L.stream>>>(p, L.partials->d(), (int)nblk);
    post(L);
    end(2);
    return -1;
  }
  long long ksplit = 1;
  if (tiles < want && p.K >= 4 * BK && L.partials) {
    ksplit = (want + tiles - 1) / tiles;
    ksplit = std::min<long long>(ksplit, (p.K + 4 * BK - 1) / (4 * BK));
    ksplit = std::min<long long>(ksplit, std::max<long long>(1, (1LL << 27) / std::max<long long>(O, 1)));
    ksplit = std::min<long long>(ksplit, 65535);
  }
  long long kchunk = (p.K + ksplit - 1) / ksplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  ksplit = (p.K + kchunk - 1) / kchunk;
  p.kchunk = kchunk;
  if (tiles > 0x7fffffffLL) throw std::runtime_error("gather_gemm: grid too large");
  if (ksplit > 1) {
    L.partials->reserve(sizeof(double) * (size_t)(ksplit * O));
    dim3 g2((unsigned)tiles, (unsigned)ksplit);
    begin();
    launch_tiled(g2, true, L.partials->d());
    post(L);
    k_reduce_partials<<<blocks_for(O, 256), 256, 0, L.stream>>>(p, L.partials->d(), (int)ksplit);
    post(L);
    end(1);
    return mixed ? -1 : shape;
  }
  dim3 grid((unsigned)tiles, 1);
  begin();
  launch_tiled(grid, false, nullptr);
  post(L);
  end(0);
  return mixed ? -1 : shape;
}

void GemmProfile::fold() {
  if (pairs.empty()) return;
  FNOCC_CUDA(cudaEventSynchronize(pool[pairs.back().second]));
  for (size_t i = 0; i < pairs.size(); ++i) {
    float t = 0;
    FNOCC_CUDA(cudaEventElapsedTime(&t, pool[pairs[i].first], pool[pairs[i].second]));
    ms[path[i]] += t;
    flop_sum[path[i]] += flops[i];
    ++launches[path[i]];
  }
  pairs.clear();
  flops.clear();
  path.clear();
}

void gather_axpy(const Launch &L, long long M, double alpha, const double *A, const DMap &arow, double *C,
                 const DMap &crow, long long asize, long long csize) {
  if (M <= 0) return;
  if (arow.maxoff >= asize || crow.maxoff >= csize || arow.maxoff < 0 || crow.maxoff < 0)
    throw std::runtime_error("gather_axpy: index map exceeds operand bounds");
  k_gather_axpy<<<blocks_for(M, 256), 256, 0, L.stream>>>(M, alpha, A, arow, C, crow);
  post(L);
}

void antisym_pack(const Launch &L, const double *Y, int nh, int np, int o, int v, const int *htab, long long nhtup,
                  const int *ptab, long long nptup, double *out, double scale, bool accumulate, bool canonical) {
  ensure_perm_tables();
  if ((o | v) & 1) throw std::runtime_error("antisym_pack: odd spin-orbital count");
  long long n = nhtup * nptup;
  if (n <= 0) return;
  k_antisym_pack<<<blocks_for(n, 256), 256, 0, L.stream>>>(Y, nh, np, o, v, htab, nhtup, ptab, nptup, out, scale,
                                                            accumulate ? 1 : 0, canonical ? 1 : 0);
  post(L);
}

// out = in with every index of a spin-orbital tensor [n^rank] (occupied
// first, then virtual) moved to its canonical position within its space
__global__ void k_canonical_layout(const double *in, int n, int o, int rank, double *out) {
  long long total = 1;
  for (int k = 0; k < rank; ++k) total *= n;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  long long rem = idx, off = 0, mul = 1;
  for (int k = 0; k < rank; ++k) {
    const int p = (int)(rem % n);
    rem /= n;
    off += mul * (p < o ? canon_pos(p, o) : o + canon_pos(p - o, n - o));
    mul *= n;
  }
  out[off] = in[idx];
}

void canonical_layout(const Launch &L, const double *in, int n, int o, int rank, double *out) {
  if ((o & 1) || ((n - o) & 1) || rank < 1 || rank > 4) throw std::runtime_error("canonical_layout: bad shape");
  long long total = 1;
  for (int k = 0; k < rank; ++k) total *= n;
  k_canonical_layout<<<blocks_for(total, 256), 256, 0, L.stream>>>(in, n, o, rank, out);
  post(L);
}

void unpack_dense_rows(const Launch &L, const double *packed, int nh, int np, int o, int v, const long long *hrank,
                       const long long *prank, long long nptup, double *dense) {
  if (np < 1 || nh > 4 || np > 4 || v > 160) throw std::runtime_error("unpack_dense_rows: unsupported sizes");
  if ((o | v) & 1) throw std::runtime_error("unpack_dense_rows: odd spin-orbital count");
  const int ni = std::min(np, 3);  // inner particles: at most v^3 elements per block
  long long outer = 1, inner = 1;
  for (int k = 0; k < nh; ++k) outer *= o;
  for (int k = 0; k < np - ni; ++k) outer *= v;
  for (int k = 0; k < ni; ++k) inner *= v;
  if (outer <= 0 || inner <= 0) return;
  if (outer > 0x7fffffffLL || inner > 0xffffffffLL) throw std::runtime_error("unpack_dense_rows: too large");
  const unsigned grid = (unsigned)outer;
#define FNOCC_U(a, b)                                                                                      \
  if (nh == a && np == b) {                                                                                \
    k_unpack_blocks<a, b><<<grid, 256, 0, L.stream>>>(packed, o, v, hrank, prank, nptup, inner, dense); \
    post(L);                                                                                               \
    return;                                                                                                \
  }
  FNOCC_U(0, 1) FNOCC_U(0, 2) FNOCC_U(1, 1) FNOCC_U(1, 2) FNOCC_U(1, 3) FNOCC_U(2, 1) FNOCC_U(2, 2)
  FNOCC_U(2, 3) FNOCC_U(2, 4) FNOCC_U(3, 1) FNOCC_U(3, 2) FNOCC_U(3, 3) FNOCC_U(4, 1) FNOCC_U(4, 2)
#undef FNOCC_U
  throw std::runtime_error("unpack_dense_rows: no kernel for this component");
}

void unpack_dense(const Launch &L, const double *packed, int nh, int np, int o, int v, const int *htab,
                  long long nhtup, const int *ptab, long long nptup, double *dense) {
  ensure_perm_tables();
  if ((o | v) & 1) throw std::runtime_error("unpack_dense: odd spin-orbital count");
  long long dn = 1;
  for (int k = 0; k < nh; ++k) dn *= o;
  for (int k = 0; k < np; ++k) dn *= v;
  FNOCC_CUDA(cudaMemsetAsync(dense, 0, dn * sizeof(double), L.stream));
  long long n = nhtup * nptup;
  if (n <= 0) return;
  k_unpack_dense<<<blocks_for(n, 256), 256, 0, L.stream>>>(packed, nh, np, o, v, htab, nhtup, ptab, nptup, dense);
  post(L);
}

void fill(const Launch &L, double *x, double val, long long n) {
  if (n <= 0) return;
  k_fill<<<blocks_for(n, 256), 256, 0, L.stream>>>(x, val, n);
  post(L);
}

void axpby(const Launch &L, long long n, double a, const double *x, double b, double *y) {
  if (n <= 0) return;
  k_axpby<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, a, x, b, y);
  post(L);
}

void scale_mask(const Launch &L, long long n, double *x, const unsigned char *mask) {
  if (n <= 0) return;
  k_scale_mask<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, x, mask);
  post(L);
}

void gather_idx(const Launch &L, long long n, const long long *idx, const double *src, double *dst) {
  if (n <= 0) return;
  k_gather_idx<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, idx, src, dst);
  post(L);
}

void scatter_idx(const Launch &L, long long n, const long long *idx, const double *src, double *dst) {
  if (n <= 0) return;
  k_scatter_idx<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, idx, src, dst);
  post(L);
}

void jacobi_update(const Launch &L, long long n, const double *r, const double *d, double *t) {
  if (n <= 0) return;
  k_jacobi_update<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, r, d, t);
  post(L);
}

void precondition(const Launch &L, long long n, const double *r, const double *d, double theta,
                  const unsigned char *mask, double *out) {
  if (n <= 0) return;
  k_precondition<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, r, d, theta, mask, out);
  post(L);
}

void multi_dot(const Launch &L, long long n, const double *x, const double *Y, long long ld, int nvec,
               double *dots_dev, DevBuf &part) {
  if (nvec <= 0) return;
  int gx = (int)std::min<long long>(std::max<long long>(1, (n + 256 * 8 - 1) / (256 * 8)), 256);
  part.reserve(sizeof(double) * (size_t)gx * nvec);
  dim3 grid(gx, nvec);
  k_dot_partial<<<grid, 256, 0, L.stream>>>(n, x, Y, ld, part.d());
  post(L);
  k_dot_final<<<blocks_for(nvec, 128), 128, 0, L.stream>>>(gx, nvec, part.d(), dots_dev);
  post(L);
}

void lincomb(const Launch &L, long long n, const double *X, long long ld, int k, const double *coef_dev, double *y,
             bool accumulate) {
  if (n <= 0) return;
  const int grid = (int)std::min<long long>(blocks_for(n, 256), (long long)L.sms * 8);
  k_lincomb<<<grid, 256, sizeof(double) * std::max(k, 1), L.stream>>>(n, X, ld, k, coef_dev, y, accumulate ? 1 : 0);
  post(L);
}

void absmax_sumsq(const Launch &L, long long n, const double *x, double *out2_dev, DevBuf &part) {
  int gx = (int)std::min<long long>(std::max<long long>(1, (n + 256 * 8 - 1) / (256 * 8)), 256);
  part.reserve(sizeof(double) * 2 * gx);
  k_absmax_partial<<<gx, 256, 0, L.stream>>>(n, x, part.d());
  post(L);
  k_absmax_final<<<1, 32, 0, L.stream>>>(gx, part.d(), out2_dev);
  post(L);
}

void spin_orbital_eri(const Launch &L, const double *eri_sp, int n, double *g) {
  long long ns = 2LL * n;
  long long tot = ns * ns * ns * ns;
  k_spin_eri<<<blocks_for(tot, 256), 256, 0, L.stream>>>(eri_sp, n, g);
  post(L);
}

void spin_orbital_h(const Launch &L, const double *h_sp, int n, double *hso) {
  int ns = 2 * n;
  k_spin_h<<<blocks_for((long long)ns * ns, 256), 256, 0, L.stream>>>(h_sp, n, hso);
  post(L);
}

void normal_order(const Launch &L, const double *h, const double *g, int n, int o, double *f, double *eref2_dev) {
  k_normal_order<<<blocks_for((long long)n * n, 256), 256, 0, L.stream>>>(h, g, n, o, f);
  post(L);
  if (eref2_dev) {
    k_eref<<<1, 256, 0, L.stream>>>(h, g, n, o, eref2_dev);
    post(L);
  }
}

void t1_transform_mats(const Launch &L, const double *t1, int o, int v, double *Lm, double *Mm) {
  int n = o + v;
  k_t1_mats<<<blocks_for((long long)n * n, 256), 256, 0, L.stream>>>(t1, o, v, Lm, Mm);
  post(L);
}

void jacobi_eig(const Launch &L, double *A, int n, double *evals, double *V, int *info_dev) {
  if (n > 128) throw std::runtime_error("jacobi_eig: n > 128");
  size_t smem = sizeof(double) * (size_t)n * n;
  {
    static std::mutex mu;
    static bool attr[64] = {false};
    int dev = 0;
    FNOCC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) throw std::runtime_error("device index out of range");
    if (!attr[dev]) {
      FNOCC_CUDA(cudaFuncSetAttribute(k_jacobi_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 8));
      attr[dev] = true;
    }
  }
  k_jacobi_eig<<<1, 512, smem, L.stream>>>(A, n, evals, V, info_dev);
  post(L);
}

void permute_columns(const Launch &L, const double *in, int rows, int cols_in, const int *perm, int cols_out,
                     double *out) {
  long long tot = (long long)rows * cols_out;
  if (tot <= 0) return;
  k_permute_columns<<<blocks_for(tot, 256), 256, 0, L.stream>>>(in, rows, cols_in, perm, cols_out, out);
  post(L);
}

void fix_phase(const Launch &L, double *c, int rows, int cols) {
  if (cols <= 0) return;
  k_fix_phase<<<blocks_for(cols, 128), 128, 0, L.stream>>>(c, rows, cols);
  post(L);
}

void lincomb3(const Launch &L, long long n, double *out, const double *a, double alpha, const double *b,
              double beta, const double *c) {
  if (n <= 0) return;
  k_lincomb3<<<blocks_for(n, 256), 256, 0, L.stream>>>(n, out, a, alpha, b, beta, c);
  post(L);
}

void mp2_amplitudes(const Launch &L, const double *g, const double *fdiag, int n, int o, double *t) {
  long long v = n - o;
  long long tot = (long long)o * o * v * v;
  if (tot <= 0) return;
  k_mp2<<<blocks_for(tot, 256), 256, 0, L.stream>>>(g, fdiag, n, o, t);
  post(L);
}

void diag_of(const Launch &L, const double *a, int n, double *d) {
  k_diag<<<blocks_for(n, 128), 128, 0, L.stream>>>(a, n, d);
  post(L);
}

void alpha_block(const Launch &L, const double *in, int nso, double *out) {
  int m = nso / 2;
  k_alpha_block<<<blocks_for((long long)m * m, 256), 256, 0, L.stream>>>(in, nso, out);
  post(L);
}

void eom_diag(const Launch &L, const double *fdiag, int o, int nh, int np, const int *htab, long long nhtup,
              const int *ptab, long long nptup, double *d) {
  long long n = nhtup * nptup;
  if (n <= 0) return;
  k_eom_diag<<<blocks_for(n, 256), 256, 0, L.stream>>>(fdiag, o, nh, np, htab, nhtup, ptab, nptup, d);
  post(L);
}

void ms_mask(const Launch &L, int nh, int np, const int *htab, long long nhtup, const int *ptab, long long nptup,
             int ms2, unsigned char *mask) {
  long long n = nhtup * nptup;
  if (n <= 0) return;
  k_ms_mask<<<blocks_for(n, 256), 256, 0, L.stream>>>(nh, np, htab, nhtup, ptab, nptup, ms2, mask);
  post(L);
}

void cc_denominators(const Launch &L, const double *fdiag, int o, int rank, const int *htab, long long nhtup,
                     const int *ptab, long long nptup, double *d) {
  long long n = nhtup * nptup;
  if (n <= 0) return;
  k_cc_den<<<blocks_for(n, 256), 256, 0, L.stream>>>(fdiag, o, rank, htab, nhtup, ptab, nptup, d);
  post(L);
}

}  // namespace fnocc
