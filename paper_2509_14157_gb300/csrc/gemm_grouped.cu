// Grouped gather-GEMM: every spin-allowed sub-GEMM of one contraction step in
// one launch.
//
// A step of a projected equation (a term of Eq. 6 for the CCSDT residual, or
// of sigma = <mu|(H-bar R)_c|0> for the EOM variants) is one contraction
// C[m, n] += alpha * sum_k A[m, k] * B[k, n] whose row, column and reduction
// indices are index tuples of the operands. Spin symmetry splits it into
// independent sub-GEMMs (tasks). Each task carries flat offset tables, one
// 64-bit element offset per row, column and reduction index, so the kernels
// read operands in place through a single table lookup per index.
//
// The CTAs of all tasks form one grid: CTA c finds its task by binary search
// over the tasks' first-CTA offsets, then its tile and reduction slice. A task
// with few tiles splits its reduction; those partial products go to a buffer
// and a second launch adds them in a fixed order, so that for a given tile
// shape the results are bitwise reproducible (no atomics). The shape itself
// may be picked from timings (see ExecEquation::autotune); another shape sums
// in another order, so autotuned FP64 results can differ in the last bits
// between runs unless the shape is fixed.
//
// On this part FP64 FMA issue is about two per clock per SM, so an FP64 tile
// is FMA-bound whatever its shape: shapes are chosen for the least padding
// (padded multiply-adds cost full time) and for enough CTAs to occupy all SMs.
// The mixed-precision kernels run the same tasks on the tensor cores as BF16
// three-slice or TF32 two-slice split products with FP32 accumulation.
#include "common.hpp"

#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <mutex>
#include <utility>

namespace fnocc {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ int find_task(const GTask *tasks, int ntasks, long long cta) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].cta_begin <= cta)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// FP64 tile kernel: threads as TY x TX (TX = 256 / TY), each a TM x TN
// micro-tile; the block covers (TY*TM) x (TX*TN) outputs; K staged BKG at a
// time through shared memory (16, or 8 for the short reductions of single
// spin blocks, e.g. K = 5, where a 16-wide K tile would pad 3.2x). The
// operand gathers of the next K tile are issued into registers before the
// products of the current one (its reduction-index offsets read one tile
// ahead into a two-slot ring), so that their latency overlaps the FMAs;
// the order of the additions is that of the K loop either way.
template <int TY, int TM, int TN, int BKG = 16>
__global__ void __launch_bounds__(NT) k_ggemm(const GTask *__restrict__ tasks, int ntasks, double alpha,
                                              const double *__restrict__ A, const double *__restrict__ B,
                                              double *__restrict__ C, double *__restrict__ part) {
  static_assert(2 * BKG <= NT, "index staging uses 2 * BKG threads");
  constexpr int TX = NT / TY, TBM = TY * TM, TBN = TX * TN;
  constexpr int PA = (TBM * BKG + NT - 1) / NT, PB = (TBN * BKG + NT - 1) / NT;  // gathers per thread
  __shared__ double As[BKG][TBM];
  __shared__ double Bs[BKG][TBN];
  __shared__ long long arow_s[TBM], crow_s[TBM], bcol_s[TBN], ccol_s[TBN], acol_s[2][BKG], brow_s[2][BKG];
  __shared__ GTask t;
  const int tid = threadIdx.x;
  const long long cta = blockIdx.x;
  if (tid == 0) t = tasks[find_task(tasks, ntasks, cta)];
  __syncthreads();
  const long long local = cta - t.cta_begin;
  const long long z = local / t.tiles, tile = local - z * t.tiles;
  const long long m0 = (tile / t.tiles_n) * TBM, n0 = (tile % t.tiles_n) * TBN;
  const long long kb = z * t.kchunk, ke = min(t.K, kb + t.kchunk);
  const bool split = t.ksplit > 1;
  for (int i = tid; i < TBM; i += NT) {
    const long long m = m0 + i;
    arow_s[i] = m < t.M ? t.arow[m] : 0;
    crow_s[i] = (!split && m < t.M) ? t.crow[m] : 0;
  }
  for (int i = tid; i < TBN; i += NT) {
    const long long n = n0 + i;
    bcol_s[i] = n < t.N ? t.bcol[n] : 0;
    ccol_s[i] = (!split && n < t.N) ? t.ccol[n] : 0;
  }
  // reduction-index offsets of the K tile at k0 into ring slot q
  auto load_tables = [&](long long k0, int q) {
    if (tid < BKG) {
      const long long k = k0 + tid;
      acol_s[q][tid] = k < ke ? t.acol[k] : 0;
    } else if (tid < 2 * BKG) {
      const long long k = k0 + tid - BKG;
      brow_s[q][tid - BKG] = k < ke ? t.brow[k] : 0;
    }
  };
  // operand elements of the K tile at k0 (0 outside the task): thread tid
  // takes elements tid, tid + NT, ... of the A tile (k fastest) and of the
  // B tile (columns fastest)
  double pa[PA], pb[PB];
  auto gather = [&](long long k0, int q) {
#pragma unroll
    for (int j = 0; j < PA; ++j) {
      const int idx = tid + j * NT;
      const int kk = idx % BKG, row = idx / BKG;
      const bool ok = idx < TBM * BKG && (m0 + row < t.M) && (k0 + kk < ke);
      pa[j] = ok ? __ldg(A + arow_s[row] + acol_s[q][kk]) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const int idx = tid + j * NT;
      const int col = idx % TBN, kk = idx / TBN;
      const bool ok = idx < TBN * BKG && (n0 + col < t.N) && (k0 + kk < ke);
      pb[j] = ok ? __ldg(B + brow_s[q][kk] + bcol_s[col]) : 0.0;
    }
  };
  const int tx = tid % TX, ty = tid / TX;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  const long long nst = ke > kb ? (ke - kb + BKG - 1) / BKG : 0;
  if (nst > 0) {
    load_tables(kb, 0);
    __syncthreads();
    gather(kb, 0);
  }
  for (long long st = 0; st < nst; ++st) {
    const long long k0 = kb + st * BKG;
    __syncthreads();  // the products of the previous tile have read As and Bs
#pragma unroll
    for (int j = 0; j < PA; ++j) {
      const int idx = tid + j * NT;
      if (idx < TBM * BKG) As[idx % BKG][idx / BKG] = pa[j];
    }
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const int idx = tid + j * NT;
      if (idx < TBN * BKG) Bs[idx / TBN][idx % TBN] = pb[j];
    }
    // slot (st + 1) & 1 was last read by the gathers issued two tiles back
    if (st + 1 < nst) load_tables(k0 + BKG, (int)((st + 1) & 1));
    __syncthreads();
    if (st + 1 < nst) gather(k0 + BKG, (int)((st + 1) & 1));  // in flight during the products below
#pragma unroll
    for (int kk = 0; kk < BKG; ++kk) {
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
  const long long MN = t.M * t.N;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long long m = m0 + ty * TM + i;
    if (m >= t.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const long long n = n0 + tx * TN + j;
      if (n >= t.N) continue;
      if (split)
        part[t.part_off + z * MN + m * t.N + n] = acc[i][j];
      else
        C[crow_s[ty * TM + i] + ccol_s[tx * TN + j]] += alpha * acc[i][j];
    }
  }
}

// FP64 -> FP32 by truncation of the significand, in integer arithmetic (the
// FP64 pipe is the scarce unit on this part). Magnitudes below the FP32
// normal range become zero; the operands of the method are far above it.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned mant = (unsigned)((b >> 29) & 0x7fffffu);
  return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

// bits of a finite FP32 value rounded to BF16, round to nearest, ties to
// even, in the upper half of the word (integer arithmetic only)
__device__ __forceinline__ unsigned bf16_rne_bits(float x) {
  const unsigned u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
}

// exact split of an FP32 value into three BF16 slices (8 significant bits
// each; every remainder is exact in FP32)
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &s0, __nv_bfloat16 &s1, __nv_bfloat16 &s2) {
  const unsigned u0 = bf16_rne_bits(x);
  const float r1 = x - __uint_as_float(u0);
  const unsigned u1 = bf16_rne_bits(r1);
  const float r2 = r1 - __uint_as_float(u1);
  s0 = __ushort_as_bfloat16((unsigned short)(u0 >> 16));
  s1 = __ushort_as_bfloat16((unsigned short)(u1 >> 16));
  s2 = __ushort_as_bfloat16((unsigned short)(bf16_rne_bits(r2) >> 16));
}

// FP32 -> TF32 (11 significant bits) rounded to nearest, ties away from
// zero, in integer arithmetic on the bit pattern (finite inputs)
__device__ __forceinline__ unsigned tf32_rna(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }

// Split products on the tensor cores (mma.sync, FP32 accumulation). A policy
// stages each FP32 operand as kSlices narrow slices, one shared-memory plane
// per slice, and runs the slice products of one K tile of 32.
//
// Bf16x3: three BF16 slices (exact), the six products with i + j <= 2 on
// m16n8k16; the dropped products are below 2^-24 of the full one.
struct Bf16x3 {
  using slice_t = __nv_bfloat16;
  static constexpr int kSlices = 3, LDS = 40;  // padded row stride (slices)
  __device__ static void stage(float x, slice_t *p, int plane) { split3(x, p[0], p[plane], p[2 * plane]); }
  template <int TBM, int TBN, int MT, int NT2>
  __device__ static void products(const slice_t *as, const slice_t *bs, int wm, int wn, int g, int tg,
                                  float (&acc)[MT][NT2][4]) {
#pragma unroll
    for (int ks = 0; ks < 32; ks += 16) {
      unsigned a[3][MT][4], b[3][NT2][2];
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const int r0 = sl * TBM + wm * MT * 16 + mt * 16 + g;
          const int c0 = ks + 2 * tg;
          a[sl][mt][0] = *reinterpret_cast<const unsigned *>(&as[r0 * LDS + c0]);
          a[sl][mt][1] = *reinterpret_cast<const unsigned *>(&as[(r0 + 8) * LDS + c0]);
          a[sl][mt][2] = *reinterpret_cast<const unsigned *>(&as[r0 * LDS + c0 + 8]);
          a[sl][mt][3] = *reinterpret_cast<const unsigned *>(&as[(r0 + 8) * LDS + c0 + 8]);
        }
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt) {
          const int n = sl * TBN + wn * NT2 * 8 + nt * 8 + g;
          b[sl][nt][0] = *reinterpret_cast<const unsigned *>(&bs[n * LDS + ks + 2 * tg]);
          b[sl][nt][1] = *reinterpret_cast<const unsigned *>(&bs[n * LDS + ks + 2 * tg + 8]);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3 - i; ++j)
#pragma unroll
          for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT2; ++nt)
              asm volatile(
                  "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                  "{%0,%1,%2,%3};\n"
                  : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
                  : "r"(a[i][mt][0]), "r"(a[i][mt][1]), "r"(a[i][mt][2]), "r"(a[i][mt][3]), "r"(b[j][nt][0]),
                    "r"(b[j][nt][1]));
    }
  }
};

// Tf32x3: two TF32 slices (hi = x rounded to 11 significant bits, lo = the
// exact remainder rounded likewise), the three products hi*hi, hi*lo, lo*hi
// on m16n8k8; slice and dropped-product errors are about 2^-21 of the full
// product.
struct Tf32x3 {
  using slice_t = unsigned;
  static constexpr int kSlices = 2, LDS = 36;  // padded row stride (words): conflict-free fragment reads
  __device__ static void stage(float x, slice_t *p, int plane) {
    const unsigned hi = tf32_rna(x);
    p[0] = hi;
    p[plane] = tf32_rna(x - __uint_as_float(hi));
  }
  template <int TBM, int TBN, int MT, int NT2>
  __device__ static void products(const slice_t *as, const slice_t *bs, int wm, int wn, int g, int tg,
                                  float (&acc)[MT][NT2][4]) {
#pragma unroll
    for (int ks = 0; ks < 32; ks += 8) {
      unsigned a[2][MT][4], b[2][NT2][2];
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const int r0 = sl * TBM + wm * MT * 16 + mt * 16 + g;
          a[sl][mt][0] = as[r0 * LDS + ks + tg];
          a[sl][mt][1] = as[(r0 + 8) * LDS + ks + tg];
          a[sl][mt][2] = as[r0 * LDS + ks + tg + 4];
          a[sl][mt][3] = as[(r0 + 8) * LDS + ks + tg + 4];
        }
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt) {
          const int n = sl * TBN + wn * NT2 * 8 + nt * 8 + g;
          b[sl][nt][0] = bs[n * LDS + ks + tg];
          b[sl][nt][1] = bs[n * LDS + ks + tg + 4];
        }
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2 - i; ++j)
#pragma unroll
          for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT2; ++nt)
              asm volatile(
                  "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                  "{%0,%1,%2,%3};\n"
                  : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
                  : "r"(a[i][mt][0]), "r"(a[i][mt][1]), "r"(a[i][mt][2]), "r"(a[i][mt][3]), "r"(b[j][nt][0]),
                    "r"(b[j][nt][1]));
    }
  }
};

// Tile of the split-product kernels: 8 warps as WM x WN, each warp MT x NT2
// mma tiles (16 x 8), so the block tile is (WM*MT*16) x (WN*NT2*8); K tile
// 32. Software pipeline: the operand gathers of K tile t+1 are in flight
// (registers) while the tensor cores work on tile t, whose slices sit in one
// of two shared-memory buffers; one barrier per K tile.
template <class S, int WM, int WN, int MT, int NT2>
struct SplitTile {
  static constexpr int TBM = WM * MT * 16, TBN = WN * NT2 * 8, TBK = 32, LDS = S::LDS;
  static constexpr int EA = TBM * TBK / NT, EB = TBN * TBK / NT;  // gathered elements per thread and tile
  static constexpr size_t kSmem = sizeof(typename S::slice_t) * 2 * S::kSlices * (TBM + TBN) * LDS;
  static_assert(WM * WN == 8, "8 warps");
  static_assert(EA * NT == TBM * TBK && EB * NT == TBN * TBK, "whole tiles per thread");
  static_assert(LDS >= TBK, "row stride covers the K tile");
};

template <class S, int WM, int WN, int MT, int NT2>
__device__ __forceinline__ void ggemm_split(const GTask *__restrict__ tasks, int ntasks, double alpha,
                                            const double *__restrict__ A, const double *__restrict__ B,
                                            double *__restrict__ C, double *__restrict__ part) {
  using T = SplitTile<S, WM, WN, MT, NT2>;
  using slice_t = typename S::slice_t;
  constexpr int TBM = T::TBM, TBN = T::TBN, TBK = T::TBK, LDS = T::LDS, EA = T::EA, EB = T::EB;
  constexpr int NS = S::kSlices;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // As[buf][slice][row][k], Bs[buf][slice][col][k]
  slice_t *As = reinterpret_cast<slice_t *>(smem_raw);
  slice_t *Bs = As + 2 * NS * TBM * LDS;
  __shared__ long long arow_s[TBM], crow_s[TBM], bcol_s[TBN], ccol_s[TBN];
  // reduction-index offsets of the K tiles in flight (a ring of three): read
  // one tile ahead, so that no operand gather waits on a table load
  __shared__ long long acol_r[3][TBK], brow_r[3][TBK];
  __shared__ GTask t;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wm = warp / WN, wn = warp % WN;
  const int g = lane >> 2, tg = lane & 3;
  const long long cta = blockIdx.x;
  if (tid == 0) t = tasks[find_task(tasks, ntasks, cta)];
  __syncthreads();
  const long long local = cta - t.cta_begin;
  const long long z = local / t.tiles, tile = local - z * t.tiles;
  const long long m0 = (tile / t.tiles_n) * TBM, n0 = (tile % t.tiles_n) * TBN;
  const long long kb = z * t.kchunk, ke = min(t.K, kb + t.kchunk);
  const bool split = t.ksplit > 1;
  for (int i = tid; i < TBM; i += NT) {
    const long long m = m0 + i;
    arow_s[i] = m < t.M ? t.arow[m] : 0;
    crow_s[i] = (!split && m < t.M) ? t.crow[m] : 0;
  }
  for (int i = tid; i < TBN; i += NT) {
    const long long n = n0 + i;
    bcol_s[i] = n < t.N ? t.bcol[n] : 0;
    ccol_s[i] = (!split && n < t.N) ? t.ccol[n] : 0;
  }
  // table entries of the K tile at k0 into ring slot q (threads 0 .. 2 TBK - 1)
  auto load_tables = [&](long long k0, int q) {
    if (tid < TBK) {
      const long long k = k0 + tid;
      acol_r[q][tid] = k < ke ? __ldg(t.acol + k) : 0;
    } else if (tid < 2 * TBK) {
      const long long k = k0 + tid - TBK;
      brow_r[q][tid - TBK] = k < ke ? __ldg(t.brow + k) : 0;
    }
  };
  load_tables(kb, 0);
  load_tables(kb + TBK, 1);
  __syncthreads();
  double ra[EA], rb[EB];
  // gathers of the K tile at k0 into registers (0 outside the task)
  auto load = [&](long long k0, int q) {
#pragma unroll
    for (int r = 0; r < EA; ++r) {
      const int idx = tid + NT * r;
      const int kk = idx % TBK, row = idx / TBK;
      const long long k = k0 + kk;
      ra[r] = (m0 + row < t.M && k < ke) ? __ldg(A + arow_s[row] + acol_r[q][kk]) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < EB; ++r) {
      const int idx = tid + NT * r;
      const int col = idx % TBN, kk = idx / TBN;
      const long long k = k0 + kk;
      rb[r] = (n0 + col < t.N && k < ke) ? __ldg(B + brow_r[q][kk] + bcol_s[col]) : 0.0;
    }
  };
  float acc[MT][NT2][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  if (kb < ke) load(kb, 0);
  int buf = 0, q = 0;
  for (long long k0 = kb; k0 < ke; k0 += TBK, buf ^= 1, q = q == 2 ? 0 : q + 1) {
    slice_t *as = As + buf * NS * TBM * LDS, *bs = Bs + buf * NS * TBN * LDS;
#pragma unroll
    for (int r = 0; r < EA; ++r) {
      const int idx = tid + NT * r;
      const int kk = idx % TBK, row = idx / TBK;
      S::stage(f64_to_f32_trunc(ra[r]), &as[row * LDS + kk], TBM * LDS);
    }
#pragma unroll
    for (int r = 0; r < EB; ++r) {
      const int idx = tid + NT * r;
      const int col = idx % TBN, kk = idx / TBN;
      S::stage(f64_to_f32_trunc(rb[r]), &bs[col * LDS + kk], TBN * LDS);
    }
    __syncthreads();
    const int q1 = q == 2 ? 0 : q + 1, q2 = q1 == 2 ? 0 : q1 + 1;
    if (k0 + TBK < ke) load(k0 + TBK, q1);  // next tile's gathers overlap this tile's products
    if (k0 + 2 * TBK < ke) load_tables(k0 + 2 * TBK, q2);
    S::template products<TBM, TBN, MT, NT2>(as, bs, wm, wn, g, tg, acc);
  }
  const long long MN = t.M * t.N;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int rl = wm * MT * 16 + mt * 16 + g + (e >= 2 ? 8 : 0);
        const int cl = wn * NT2 * 8 + nt * 8 + 2 * tg + (e & 1);
        const long long m = m0 + rl, n = n0 + cl;
        if (m >= t.M || n >= t.N) continue;
        if (split)
          part[t.part_off + z * MN + m * t.N + n] = (double)acc[mt][nt][e];
        else
          C[crow_s[rl] + ccol_s[cl]] += alpha * (double)acc[mt][nt][e];
      }
}

template <int WM, int WN, int MT, int NT2>
__global__ void __launch_bounds__(NT) k_ggemm_bf16x3(const GTask *__restrict__ tasks, int ntasks, double alpha,
                                                     const double *__restrict__ A, const double *__restrict__ B,
                                                     double *__restrict__ C, double *__restrict__ part) {
  ggemm_split<Bf16x3, WM, WN, MT, NT2>(tasks, ntasks, alpha, A, B, C, part);
}

template <int WM, int WN, int MT, int NT2>
__global__ void __launch_bounds__(NT) k_ggemm_tf32x3(const GTask *__restrict__ tasks, int ntasks, double alpha,
                                                     const double *__restrict__ A, const double *__restrict__ B,
                                                     double *__restrict__ C, double *__restrict__ part) {
  ggemm_split<Tf32x3, WM, WN, MT, NT2>(tasks, ntasks, alpha, A, B, C, part);
}

// dynamic shared memory above the 48 KiB default, opted in once per device
// and kernel
template <class S, int WM, int WN, int MT, int NT2>
void launch_split(void (*kernel)(const GTask *, int, double, const double *, const double *, double *, double *),
                  unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha, const double *A,
                  const double *B, double *C, double *part) {
  constexpr size_t smem = SplitTile<S, WM, WN, MT, NT2>::kSmem;
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  FNOCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw std::runtime_error("grouped_gemm: device index out of range");
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
      FNOCC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      done[dev] = true;
    }
  }
  kernel<<<grid, NT, smem, s>>>(tasks, ntasks, alpha, A, B, C, part);
}

template <int WM, int WN, int MT, int NT2>
void launch_tensor(int precision, unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha,
                   const double *A, const double *B, double *C, double *part) {
  if (precision == 2)
    launch_split<Tf32x3, WM, WN, MT, NT2>(k_ggemm_tf32x3<WM, WN, MT, NT2>, grid, s, tasks, ntasks, alpha, A, B, C,
                                          part);
  else
    launch_split<Bf16x3, WM, WN, MT, NT2>(k_ggemm_bf16x3<WM, WN, MT, NT2>, grid, s, tasks, ntasks, alpha, A, B, C,
                                          part);
}

// C[crow(m) + ccol(n)] += alpha * sum_z part[task][z][m, n], z in order, for
// the tasks whose reduction was split
__global__ void k_greduce(const GTask *__restrict__ tasks, const int *__restrict__ split_ids, int nsplit,
                          long long nred, double alpha, const double *__restrict__ part, double *__restrict__ C) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= nred) return;
  int lo = 0, hi = nsplit - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tasks[split_ids[mid]].red_begin <= idx)
      lo = mid;
    else
      hi = mid - 1;
  }
  const GTask &t = tasks[split_ids[lo]];
  const long long local = idx - t.red_begin;
  const long long m = local / t.N, n = local - m * t.N;
  const long long MN = t.M * t.N;
  double s = 0.0;
  for (int z = 0; z < t.ksplit; ++z) s += part[t.part_off + z * MN + local];
  C[t.crow[m] + t.ccol[n]] += alpha * s;
}

// (TY, TM, TN, K tile) of the FP64 shapes; the last five repeat shapes 0,
// 6, 8, 11 and 12 with a K tile of 8
constexpr int kShapeDims[kGShapes][4] = {
    {16, 4, 4, 16}, {16, 8, 2, 16}, {16, 2, 8, 16}, {16, 8, 1, 16}, {16, 1, 8, 16}, {16, 2, 2, 16},
    {16, 1, 1, 16}, {64, 2, 1, 16}, {256, 1, 1, 16}, {4, 1, 2, 16},  {8, 1, 4, 16},  {2, 1, 1, 16},
    {32, 1, 1, 16}, {128, 1, 1, 16}, {16, 4, 4, 8},  {16, 1, 1, 8},  {256, 1, 1, 8}, {2, 1, 1, 8},
    {32, 1, 1, 8}};
// (WM, WN, MT, NT2) of the BF16x3 shapes: 64x64, 32x32, 128x16, 16x128, 64x16, 16x64
constexpr int kBf16Dims[kGShapesBf16][4] = {{2, 4, 2, 2}, {2, 4, 1, 1}, {8, 1, 1, 2},
                                            {1, 8, 1, 2}, {4, 2, 1, 1}, {1, 8, 1, 1}};

inline unsigned blocks_for(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

// Launchers of every shape, instantiated from the two tables above so that a
// shape's index and its template arguments cannot drift apart.
using ShapeLaunch = void (*)(unsigned, cudaStream_t, const GTask *, int, double, const double *, const double *,
                             double *, double *);
using SplitShapeLaunch = void (*)(int, unsigned, cudaStream_t, const GTask *, int, double, const double *,
                                  const double *, double *, double *);

template <int I>
void launch_fp64_shape(unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha, const double *A,
                       const double *B, double *C, double *part) {
  k_ggemm<kShapeDims[I][0], kShapeDims[I][1], kShapeDims[I][2], kShapeDims[I][3]>
      <<<grid, NT, 0, s>>>(tasks, ntasks, alpha, A, B, C, part);
}

template <int I>
void launch_split_shape(int precision, unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha,
                        const double *A, const double *B, double *C, double *part) {
  launch_tensor<kBf16Dims[I][0], kBf16Dims[I][1], kBf16Dims[I][2], kBf16Dims[I][3]>(precision, grid, s, tasks,
                                                                                     ntasks, alpha, A, B, C, part);
}

template <size_t... I>
constexpr std::array<ShapeLaunch, sizeof...(I)> fp64_launchers(std::index_sequence<I...>) {
  return {{&launch_fp64_shape<(int)I>...}};
}
template <size_t... I>
constexpr std::array<SplitShapeLaunch, sizeof...(I)> split_launchers(std::index_sequence<I...>) {
  return {{&launch_split_shape<(int)I>...}};
}

constexpr auto kFp64Launch = fp64_launchers(std::make_index_sequence<kGShapes>{});
constexpr auto kSplitLaunch = split_launchers(std::make_index_sequence<kGShapesBf16>{});

}  // namespace

void grouped_shape(int shape, int *tbm, int *tbn, int *tbk) {
  if (shape >= kGShapeTcp && shape < kGShapesAll) {
    tc_shape(shape - kGShapeTcp, tbm, tbn, tbk);
    *tbk = 16;  // one K step of the panels
    return;
  }
  if (shape >= kGShapeTc && shape < kGShapeTcp) {
    tc_shape(shape - kGShapeTc, tbm, tbn, tbk);
    return;
  }
  if (shape >= kGShapeBf16 && shape < kGShapeTc) {
    const int *d = kBf16Dims[shape - kGShapeBf16];
    *tbm = d[0] * d[2] * 16;
    *tbn = d[1] * d[3] * 8;
    *tbk = 32;
    return;
  }
  if (shape < 0 || shape >= kGShapes) throw std::runtime_error("grouped_shape: bad shape");
  const int ty = kShapeDims[shape][0], tx = NT / ty;
  *tbm = ty * kShapeDims[shape][1];
  *tbn = tx * kShapeDims[shape][2];
  *tbk = kShapeDims[shape][3];
}

void grouped_gemm(const Launch &L, const GroupedLaunch &g, double alpha, const double *A, const double *B, double *C) {
  if (g.ntasks <= 0 || g.ncta <= 0) return;
  if (g.ncta > 0x7fffffffLL) throw std::runtime_error("grouped_gemm: grid too large");
  double *part = nullptr;
  if (g.nsplit > 0) {
    if (!L.partials) throw std::runtime_error("grouped_gemm: no partial-sum scratch");
    L.partials->reserve(sizeof(double) * (size_t)g.part_need);
    part = L.partials->d();
  }
  GemmProfile *pr = (L.prof && L.prof->enabled) ? L.prof : nullptr;
  int e0 = -1;
  if (pr) {
    while (pr->pool.size() < 2 * pr->pairs.size() + 2) {
      cudaEvent_t ev;
      FNOCC_CUDA(cudaEventCreate(&ev));
      pr->pool.push_back(ev);
    }
    e0 = (int)(2 * pr->pairs.size());
    FNOCC_CUDA(cudaEventRecord(pr->pool[e0], L.stream));
  }
  const unsigned grid = (unsigned)g.ncta;
  if (g.shape >= 0 && g.shape < kGShapes)
    kFp64Launch[g.shape](grid, L.stream, g.tasks, g.ntasks, alpha, A, B, C, part);
  else if (g.shape >= kGShapeBf16 && g.shape < kGShapeTc)
    kSplitLaunch[g.shape - kGShapeBf16](L.precision, grid, L.stream, g.tasks, g.ntasks, alpha, A, B, C, part);
  else if (g.shape >= kGShapeTc && g.shape < kGShapeTcp && L.precision == 1)
    grouped_gemm_tc(g.shape - kGShapeTc, grid, L.stream, g.tasks, g.ntasks, alpha, A, B, C, part);
  else if (g.shape >= kGShapeTcp && g.shape < kGShapesAll && L.precision == 1) {
    if (!L.panels) throw std::runtime_error("grouped_gemm: no panel buffer");
    L.panels->reserve((size_t)std::max<long long>(g.panel_bytes, 256));
    grouped_gemm_tcp(g.shape - kGShapeTcp, grid, g.pack_blocks, L.stream, g.tasks, g.ntasks, alpha, A, B, C, part,
                     L.panels->as<unsigned char>());
  }
  else
    throw std::runtime_error("grouped_gemm: bad shape");
  FNOCC_CUDA(cudaGetLastError());
  if (L.counter) ++*L.counter;
  if (g.nsplit > 0) {
    k_greduce<<<blocks_for(g.nred, 256), 256, 0, L.stream>>>(g.tasks, g.split_ids, g.nsplit, g.nred, alpha, part, C);
    FNOCC_CUDA(cudaGetLastError());
    if (L.counter) ++*L.counter;
  }
  if (pr) {
    FNOCC_CUDA(cudaEventRecord(pr->pool[e0 + 1], L.stream));
    pr->pairs.push_back({e0, e0 + 1});
    pr->flops.push_back(g.flops);
    const int kind = shape_kind(g.shape);
    const int base = kind == 0 ? 0 : (kind == 3 ? 10 : (kind == 2 ? 8 : (L.precision == 2 ? 6 : 4)));
    pr->path.push_back(base + (g.nsplit > 0 ? 1 : 0));
    if (pr->pairs.size() >= 4096) pr->fold();
  }
}

}  // namespace fnocc
