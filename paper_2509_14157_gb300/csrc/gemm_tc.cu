// Grouped split-product GEMM on the fifth-generation tensor cores (tcgen05,
// accumulator in tensor memory).
//
// Same tasks as the other grouped kernels (one spin-allowed sub-GEMM of a
// contraction step per task, operands read in place through flat offset
// tables, gemm_grouped.cu), same BF16 three-slice arithmetic as the
// mixed-precision path of the single- and double-precision algorithms of
// Sec. 1: every FP64 operand element is truncated to FP32 and split exactly
// into three BF16 slices x = s0 + s1 + s2; the six slice products with
// i + j <= 2 accumulate in FP32 (the three dropped ones are below 2^-24 of
// the full product).
//
// A CTA computes a 128 x BN output tile (BN = 64, 128 or 256) in a tensor-
// memory accumulator of BN FP32 columns. K advances 32 at a time through two
// shared-memory stages. Per stage, all 256 threads gather the FP64 operand
// panels (128 x 32 of A, BN x 32 of B) through the offset tables, convert
// and split them, and store the three BF16 planes of each in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices; adjacent
// core matrices along K 128 bytes apart, along M / N 256 bytes apart); then
// one thread issues 2 K-steps x 6 slice products of tcgen05.mma kind::f16
// (M = 128, N = BN, K = 16) and commits them to the stage's mbarrier, which
// frees the stage two iterations later. The gathers of the next stage are in
// flight while the tensor cores work on the current one. The epilogue reads
// the accumulator with tcgen05.ld (warp w reads lanes 32 (w mod 4) .. +31,
// half of the columns each), converts to FP64 and scatters C[crow + ccol] +=
// alpha * acc, or writes a split-reduction partial.
//
// Every wait on an mbarrier is bounded (about 2 s of SM clock); on expiry
// the kernel records a status word that the host reads after the product
// (fnocc returns FNOCC_E_TIMEOUT), skips the output, waits (bounded) for its
// own committed products, frees its tensor memory and returns.
#include "common.hpp"

#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

namespace fnocc {

namespace {

constexpr int kThreads = 256;
constexpr int kBM = 128;  // accumulator lanes
constexpr int kBK = 32;   // K per stage: two K-steps of the f16 kind
constexpr long long kTimeoutCycles = 4000000000LL;  // about 2 s at 2 GHz

// status word of the last bounded wait that expired (0 = none), per device
__device__ int g_tc_status;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

// true when the phase with the given parity has completed, false after the
// time limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long start = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - start > kTimeoutCycles) return false;
  }
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle;
// lbo / sbo: byte distance of adjacent core matrices along K / along M or N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int find_task_tc(const GTask *tasks, int ntasks, long long cta) {
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

// FP64 -> FP32 by truncation of the significand (integer arithmetic); then
// an exact three-way BF16 split
__device__ __forceinline__ float trunc_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// bits of a finite FP32 value rounded to BF16 (8 significant bits), round
// to nearest, ties to even, kept in the upper half of the word: integer
// arithmetic only (no conversion unit)
__device__ __forceinline__ uint32_t bf16_rne_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
}

// x = s0 + s1 + s2 exactly (24 = 3 x 8 significant bits; each remainder is
// exact in FP32); the BF16 slices as their 16-bit patterns
__device__ __forceinline__ void split3(double xd, uint16_t &s0, uint16_t &s1, uint16_t &s2) {
  const float x = trunc_f32(xd);
  const uint32_t u0 = bf16_rne_bits(x);
  const float r1 = x - __uint_as_float(u0);
  const uint32_t u1 = bf16_rne_bits(r1);
  const float r2 = r1 - __uint_as_float(u1);
  s0 = (uint16_t)(u0 >> 16);
  s1 = (uint16_t)(u1 >> 16);
  s2 = (uint16_t)(bf16_rne_bits(r2) >> 16);
}

// byte offset of element (row, k) of a K-step plane (k < 16): core matrix
// (row / 8, k / 8), 16-byte row (row % 8), element k % 8
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int BN>
struct TcTile {
  static constexpr int kPlaneA = kBM * 16 * 2;  // bytes of one K-step plane of A
  static constexpr int kPlaneB = BN * 16 * 2;
  static constexpr int kStageA = 3 * 2 * kPlaneA;  // three slices x two K-steps
  static constexpr int kStageB = 3 * 2 * kPlaneB;
  static constexpr int kStage = kStageA + kStageB;
  static constexpr size_t kSmem = 2 * (size_t)kStage + 1024;  // two stages + alignment slack
  static constexpr int EA = kBM * kBK / kThreads;  // gathered A elements per thread and stage
  static constexpr int EB = BN * kBK / kThreads;
  static_assert(EA % 2 == 0 && EB % 2 == 0 && kBM * kBK / 64 == 8 * (EA / 2) && BN * kBK / 64 == 8 * (EB / 2),
                "every core matrix of a stage taken by exactly one warp");
  static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "accumulator width");
};

// TR = false: the accumulator lanes (the tcgen05 M dimension) run over the
// 128 rows of an A tile and its columns over BN columns of B; TR = true (for
// steps with few rows): lanes over 128 columns of B and columns over BN
// rows of A, i.e. the tile of C is computed transposed in tensor memory.
// X is the operand on the lanes, Y the one on the columns.
template <int BN, bool TR>
__global__ void __launch_bounds__(kThreads, BN <= 128 ? 2 : 1)
    k_ggemm_tc(const GTask *__restrict__ tasks, int ntasks, double alpha, const double *__restrict__ A,
               const double *__restrict__ B, double *__restrict__ C, double *__restrict__ part) {
  using T = TcTile<BN>;
  constexpr int EA = T::EA, EB = T::EB;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ long long xrow_s[kBM], cx_s[kBM], yrow_s[BN], cy_s[BN];
  // reduction-index offsets of the K tiles kt, kt + 1, kt + 2 (a ring): read
  // one stage ahead, so that no operand gather waits on a table load
  __shared__ long long xk_r[3][kBK], yk_r[3][kBK];
  __shared__ GTask t;
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long cta = blockIdx.x;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_s)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    t = tasks[find_task_tc(tasks, ntasks, cta)];
    abort_s = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const long long local = cta - t.cta_begin;
  const long long z = local / t.tiles, tile = local - z * t.tiles;
  // tile order: n fastest (consecutive CTAs share the A row tile), or m
  // fastest where B is the larger operand (they share its column tile in L2)
  const long long tiles_m = t.tiles / t.tiles_n;
  constexpr int TBM = TR ? BN : kBM, TBN = TR ? kBM : BN;
  const long long m0 = (t.mfast ? tile % tiles_m : tile / t.tiles_n) * TBM,
                  n0 = (t.mfast ? tile / tiles_m : tile % t.tiles_n) * TBN;
  const long long x0 = TR ? n0 : m0, y0 = TR ? m0 : n0;  // first X and Y index of the tile
  const long long XN = TR ? t.N : t.M, YN = TR ? t.M : t.N;
  const long long *xrow = TR ? t.bcol : t.arow, *yrow = TR ? t.arow : t.bcol;
  const long long *cxt = TR ? t.ccol : t.crow, *cyt = TR ? t.crow : t.ccol;
  const long long *xkt = TR ? t.brow : t.acol, *ykt = TR ? t.acol : t.brow;
  const double *X = TR ? B : A, *Y = TR ? A : B;
  const long long kb = z * t.kchunk, ke = min(t.K, kb + t.kchunk);
  const bool split = t.ksplit > 1;
  for (int i = tid; i < kBM; i += kThreads) {
    const long long x = x0 + i;
    xrow_s[i] = x < XN ? xrow[x] : 0;
    cx_s[i] = (!split && x < XN) ? cxt[x] : 0;
  }
  for (int i = tid; i < BN; i += kThreads) {
    const long long y = y0 + i;
    yrow_s[i] = y < YN ? yrow[y] : 0;
    cy_s[i] = (!split && y < YN) ? cyt[y] : 0;
  }
  // table entries of the K tile at k0 into ring slot q (threads 0 .. 2 kBK - 1)
  auto load_tables = [&](long long k0, int q) {
    if (tid < kBK) {
      const long long k = k0 + tid;
      xk_r[q][tid] = k < ke ? __ldg(xkt + k) : 0;
    } else if (tid < 2 * kBK) {
      const long long k = k0 + tid - kBK;
      yk_r[q][tid - kBK] = k < ke ? __ldg(ykt + k) : 0;
    }
  };
  load_tables(kb, 0);
  load_tables(kb + kBK, 1);
  __syncthreads();

  double ra[EA], rb[EB];
  // Gathers of the stage at k0 into registers (0 outside the task). The
  // stage's operand planes are sets of core matrices (8 rows x 8 k): A has
  // 16 row groups x 4 k chunks, B has BN / 8 column groups x 4 k chunks, and
  // warp w takes core matrices w, w + 8, w + 16, ...; lane l takes row l / 4
  // of the core matrix and its k pair 2 (l mod 4), 2 (l mod 4) + 1, so that
  // each later store of a warp fills one core matrix's 128 contiguous bytes
  // (no bank conflict).
  auto load = [&](long long k0, int q) {
#pragma unroll
    for (int j = 0; j < EA / 2; ++j) {
      const int cm = warp + 8 * j, rg = cm & 15, kc = cm >> 4;
      const int row = rg * 8 + (lane >> 2), kk = kc * 8 + 2 * (lane & 3);
      const bool rok = x0 + row < XN;
      ra[2 * j] = (rok && k0 + kk < ke) ? __ldg(X + xrow_s[row] + xk_r[q][kk]) : 0.0;
      ra[2 * j + 1] = (rok && k0 + kk + 1 < ke) ? __ldg(X + xrow_s[row] + xk_r[q][kk + 1]) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < EB / 2; ++j) {
      const int cm = warp + 8 * j, cg = cm % (BN / 8), kc = cm / (BN / 8);
      const int col = cg * 8 + (lane >> 2), kk = kc * 8 + 2 * (lane & 3);
      const bool cok = y0 + col < YN;
      rb[2 * j] = (cok && k0 + kk < ke) ? __ldg(Y + yk_r[q][kk] + yrow_s[col]) : 0.0;
      rb[2 * j + 1] = (cok && k0 + kk + 1 < ke) ? __ldg(Y + yk_r[q][kk + 1] + yrow_s[col]) : 0.0;
    }
  };

  const long long nk = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;
  const uint32_t sbase = smem_u32(smem);
  constexpr uint32_t idesc = idesc_bf16(kBM, BN);
  // the six slice products i + j <= 2 (A slice i, B slice j)
  constexpr int kPi[6] = {0, 0, 1, 0, 1, 2}, kPj[6] = {0, 1, 0, 2, 1, 0};
  if (nk > 0) load(kb, 0);
  for (long long kt = 0; kt < nk; ++kt) {
    const int s = (int)(kt & 1);
    unsigned char *stA = smem + s * T::kStage;
    unsigned char *stB = stA + T::kStageA;
    if (kt >= 2) {  // the products of stage s two iterations back have read it
      if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((kt - 2) >> 1) & 1))) abort_s = 1;
      __syncthreads();
      if (abort_s) break;
    }
    // the three slices of each element pair as 32-bit words (element k in
    // the low half), one core-matrix row chunk per lane
#pragma unroll
    for (int j = 0; j < EA / 2; ++j) {
      const int cm = warp + 8 * j, rg = cm & 15, kc = cm >> 4;
      uint16_t a0, a1, a2, b0, b1, b2;
      split3(ra[2 * j], a0, a1, a2);
      split3(ra[2 * j + 1], b0, b1, b2);
      const uint32_t off = (uint32_t)((kc >> 1) * T::kPlaneA + rg * 256 + (kc & 1) * 128 + (lane >> 2) * 16 +
                                      (lane & 3) * 4);
      *reinterpret_cast<uint32_t *>(stA + off) = (uint32_t)a0 | ((uint32_t)b0 << 16);
      *reinterpret_cast<uint32_t *>(stA + 2 * T::kPlaneA + off) = (uint32_t)a1 | ((uint32_t)b1 << 16);
      *reinterpret_cast<uint32_t *>(stA + 4 * T::kPlaneA + off) = (uint32_t)a2 | ((uint32_t)b2 << 16);
    }
#pragma unroll
    for (int j = 0; j < EB / 2; ++j) {
      const int cm = warp + 8 * j, cg = cm % (BN / 8), kc = cm / (BN / 8);
      uint16_t a0, a1, a2, b0, b1, b2;
      split3(rb[2 * j], a0, a1, a2);
      split3(rb[2 * j + 1], b0, b1, b2);
      const uint32_t off = (uint32_t)((kc >> 1) * T::kPlaneB + cg * 256 + (kc & 1) * 128 + (lane >> 2) * 16 +
                                      (lane & 3) * 4);
      *reinterpret_cast<uint32_t *>(stB + off) = (uint32_t)a0 | ((uint32_t)b0 << 16);
      *reinterpret_cast<uint32_t *>(stB + 2 * T::kPlaneB + off) = (uint32_t)a1 | ((uint32_t)b1 << 16);
      *reinterpret_cast<uint32_t *>(stB + 4 * T::kPlaneB + off) = (uint32_t)a2 | ((uint32_t)b2 << 16);
    }
    // generic-proxy stores become visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (kt + 1 < nk) load(kb + (kt + 1) * kBK, (int)((kt + 1) % 3));  // in flight during the products below
    if (kt + 2 < nk) load_tables(kb + (kt + 2) * kBK, (int)((kt + 2) % 3));
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = sbase + s * T::kStage, b0 = a0 + T::kStageA;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint64_t ad = smem_desc(a0 + (kPi[p] * 2 + ks) * T::kPlaneA, 128, 256);
          const uint64_t bd = smem_desc(b0 + (kPj[p] * 2 + ks) * T::kPlaneB, 128, 256);
          mma_bf16(tmem, ad, bd, idesc, (kt > 0 || ks > 0 || p > 0) ? 1u : 0u);
        }
      mma_commit(smem_u32(&mbar[s]));
    }
  }
  bool ok = !abort_s;
  if (ok && nk > 0) {
    const long long last = nk - 1;
    if (!mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1))) ok = false;
  }
  if (!ok) {
    if (tid == 0) atomicExch(&g_tc_status, 1);
    // let products already committed finish (bounded) before the memory goes
    if (nk > 0) {
      const long long last = nk - 1;
      mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int q = warp & 3, half = warp >> 2;
    const int rl = q * 32 + lane;
    const long long x = x0 + rl;
    const long long MN = t.M * t.N;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      const int cl0 = half * (BN / 2) + c * 16;
      float v[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cl0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (x >= XN) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const long long y = y0 + cl0 + i;
        if (y >= YN) break;
        if (split)
          part[t.part_off + z * MN + (TR ? y * t.N + x : x * t.N + y)] = (double)v[i];
        else
          C[cx_s[rl] + cy_s[cl0 + i]] += alpha * (double)v[i];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

template <int BN, bool TR>
void launch_tc(unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha, const double *A,
               const double *B, double *C, double *part) {
  constexpr size_t smem = TcTile<BN>::kSmem;
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  FNOCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw std::runtime_error("grouped_gemm_tc: device index out of range");
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
      FNOCC_CUDA(cudaFuncSetAttribute(k_ggemm_tc<BN, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      done[dev] = true;
    }
  }
  k_ggemm_tc<BN, TR><<<grid, kThreads, smem, s>>>(tasks, ntasks, alpha, A, B, C, part);
}


// ---------------------------------------------------------------------------
// Panel form: the operands of a step are gathered, truncated and split once
// per step into BF16 panels laid out as the tensor cores read them, then a
// GEMM kernel streams the panels into shared memory with bulk copies (TMA,
// cp.async.bulk) through a ring of stages, one thread issuing the copies,
// one thread issuing the products, all four warps draining the accumulator.
// A panel block is one 16-wide K step of one tile: three BF16 slices, each
// a K-step plane in the canonical K-major layout (core matrices 128 bytes
// apart along K, 256 bytes along rows), so a stage is two contiguous copies.
// ---------------------------------------------------------------------------

constexpr int kPackThreads = 256;
constexpr int kTcpThreads = 128;

template <int BN>
struct TcpTile {
  static constexpr int kBlockA = 3 * kBM * 16 * 2;   // bytes of one A panel block (three slices)
  static constexpr int kBlockB = 3 * BN * 16 * 2;
  static constexpr int kStage = kBlockA + kBlockB;
  static constexpr int kStages = BN >= 256 ? 5 : 4;   // 180 KiB / 96 KiB / 72 KiB of stages
  static constexpr size_t kSmem = (size_t)kStages * kStage + 1024;
};

__device__ __forceinline__ int find_pack_task(const GTask *tasks, int ntasks, long long blk) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].pk_begin <= blk)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One CTA per panel block: rows R (128 for A, BN for B) x 16 K of the task,
// zero outside it, split into the three slice planes of the block.
template <int BN>
__global__ void __launch_bounds__(kPackThreads) k_tc_pack(const GTask *__restrict__ tasks, int ntasks,
                                                          const double *__restrict__ A,
                                                          const double *__restrict__ B,
                                                          unsigned char *__restrict__ panels) {
  __shared__ long long rowoff[BN > kBM ? BN : kBM];
  __shared__ long long koff[16];
  __shared__ GTask t;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long blk = blockIdx.x;
  if (tid == 0) t = tasks[find_pack_task(tasks, ntasks, blk)];
  __syncthreads();
  const long long tiles_m = t.tiles / t.tiles_n;
  long long local = blk - t.pk_begin;
  const bool isA = local < tiles_m * t.ksteps;
  if (!isA) local -= tiles_m * t.ksteps;
  const long long tile = local / t.ksteps, ks = local - tile * t.ksteps;
  const int R = isA ? kBM : BN;
  const long long r0 = tile * R, k0 = ks * 16;
  const long long nrows = isA ? t.M : t.N;
  for (int i = tid; i < R; i += kPackThreads) {
    const long long r = r0 + i;
    rowoff[i] = r < nrows ? (isA ? t.arow[r] : t.bcol[r]) : -1;
  }
  if (tid < 16) {
    const long long k = k0 + tid;
    koff[tid] = k < t.K ? (isA ? t.acol[k] : t.brow[k]) : -1;
  }
  __syncthreads();
  const double *src = isA ? A : B;
  unsigned char *dst = panels + (isA ? t.apanel + (tile * t.ksteps + ks) * (long long)TcpTile<BN>::kBlockA
                                     : t.bpanel + (tile * t.ksteps + ks) * (long long)TcpTile<BN>::kBlockB);
  const int plane = R * 32;  // bytes of one slice plane
  // core matrices (R / 8 row groups x 2 k chunks); warp w takes w, w + 8, ...;
  // lane l: row l / 4 of the core matrix, k pair 2 (l mod 4), 2 (l mod 4) + 1
  for (int cm = warp; cm < R / 4; cm += kPackThreads / 32) {
    const int rg = cm >> 1, kc = cm & 1;
    const int r = rg * 8 + (lane >> 2), kk = kc * 8 + 2 * (lane & 3);
    double x0 = 0.0, x1 = 0.0;
    const long long ro = rowoff[r];
    if (ro >= 0) {
      if (koff[kk] >= 0) x0 = __ldg(src + ro + koff[kk]);
      if (koff[kk + 1] >= 0) x1 = __ldg(src + ro + koff[kk + 1]);
    }
    uint16_t a0, a1, a2, b0, b1, b2;
    split3(x0, a0, a1, a2);
    split3(x1, b0, b1, b2);
    const int off = rg * 256 + kc * 128 + (lane >> 2) * 16 + (lane & 3) * 4;
    *reinterpret_cast<uint32_t *>(dst + off) = (uint32_t)a0 | ((uint32_t)b0 << 16);
    *reinterpret_cast<uint32_t *>(dst + plane + off) = (uint32_t)a1 | ((uint32_t)b1 << 16);
    *reinterpret_cast<uint32_t *>(dst + 2 * plane + off) = (uint32_t)a2 | ((uint32_t)b2 << 16);
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// bulk copy global -> shared, completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kTcpThreads, 1)
    k_ggemm_tcp(const GTask *__restrict__ tasks, int ntasks, double alpha, double *__restrict__ C,
                double *__restrict__ part, const unsigned char *__restrict__ panels) {
  using T = TcpTile<BN>;
  constexpr int S = T::kStages;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ long long crow_s[kBM], ccol_s[BN];
  __shared__ GTask t;
  __shared__ __align__(8) unsigned long long full[S], empty[S], done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long cta = blockIdx.x;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_s)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    t = tasks[find_task_tc(tasks, ntasks, cta)];
    abort_s = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const long long local = cta - t.cta_begin;
  const long long z = local / t.tiles, tile = local - z * t.tiles;
  const long long tiles_m = t.tiles / t.tiles_n;
  const long long mt = t.mfast ? tile % tiles_m : tile / t.tiles_n, nt = t.mfast ? tile / tiles_m : tile % t.tiles_n;
  const long long m0 = mt * kBM, n0 = nt * BN;
  const bool split = t.ksplit > 1;
  for (int i = tid; i < kBM; i += kTcpThreads) {
    const long long m = m0 + i;
    crow_s[i] = (!split && m < t.M) ? t.crow[m] : 0;
  }
  for (int i = tid; i < BN; i += kTcpThreads) {
    const long long n = n0 + i;
    ccol_s[i] = (!split && n < t.N) ? t.ccol[n] : 0;
  }
  __syncthreads();
  // K steps of this CTA (the reduction chunk is a whole number of steps)
  const long long ks0 = (z * t.kchunk) / 16;
  const long long ks1 = min((long long)t.ksteps, ((z + 1) * t.kchunk + 15) / 16);
  const long long nk = ks1 > ks0 ? ks1 - ks0 : 0;
  const uint32_t sbase = smem_u32(smem);
  constexpr uint32_t idesc = idesc_bf16(kBM, BN);
  constexpr int kPi[6] = {0, 0, 1, 0, 1, 2}, kPj[6] = {0, 1, 0, 2, 1, 0};
  if (tid == 0 && nk > 0) {  // producer: bulk copies of the panel blocks into the ring
    const unsigned char *pa = panels + t.apanel + (mt * t.ksteps + ks0) * (long long)T::kBlockA;
    const unsigned char *pb = panels + t.bpanel + (nt * t.ksteps + ks0) * (long long)T::kBlockB;
    long long it = 0;
    for (; it < nk; ++it) {
      const int s = (int)(it % S);
      if (it >= S && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((it / S) - 1) & 1))) {
        abort_s = 1;
        break;
      }
      if (*(volatile int *)&abort_s) break;
      const uint32_t a_dst = sbase + s * T::kStage, b_dst = a_dst + T::kBlockA;
      mbar_expect_tx(smem_u32(&full[s]), (uint32_t)T::kStage);
      bulk_g2s(a_dst, pa + it * T::kBlockA, (uint32_t)T::kBlockA, smem_u32(&full[s]));
      bulk_g2s(b_dst, pb + it * T::kBlockB, (uint32_t)T::kBlockB, smem_u32(&full[s]));
    }
    if (it < nk && it > 0) {  // stopped early: copies already issued land before the memory goes
      const long long last = it - 1;
      mbar_wait(smem_u32(&full[last % S]), (uint32_t)((last / S) & 1));
    }
  } else if (tid == 32 && nk > 0) {  // products
    long long it = 0;
    for (; it < nk; ++it) {
      const int s = (int)(it % S);
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((it / S) & 1)) || *(volatile int *)&abort_s) {
        abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = sbase + s * T::kStage, b0 = a0 + T::kBlockA;
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const uint64_t ad = smem_desc(a0 + kPi[p] * (kBM * 32), 128, 256);
        const uint64_t bd = smem_desc(b0 + kPj[p] * (BN * 32), 128, 256);
        mma_bf16(tmem, ad, bd, idesc, (it > 0 || p > 0) ? 1u : 0u);
      }
      mma_commit(smem_u32(&empty[s]));
    }
    mma_commit(smem_u32(&done));  // arrives once every product issued above has completed
  }
  __syncwarp();
  bool ok = true;
  if (nk > 0 && !mbar_wait(smem_u32(&done), 0u)) ok = false;
  __syncthreads();
  if (abort_s) ok = false;
  if (!ok) {
    if (tid == 0) atomicExch(&g_tc_status, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int rl = warp * 32 + lane;  // accumulator lane = output row
    const long long m = m0 + rl;
    const long long MN = t.M * t.N;
#pragma unroll 1
    for (int c = 0; c < BN / 16; ++c) {
      float v[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (m >= t.M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const long long n = n0 + c * 16 + i;
        if (n >= t.N) break;
        if (split)
          part[t.part_off + z * MN + m * t.N + n] = (double)v[i];
        else
          C[crow_s[rl] + ccol_s[c * 16 + i]] += alpha * (double)v[i];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

template <int BN>
void launch_tcp(unsigned grid, long long pack_blocks, cudaStream_t s, const GTask *tasks, int ntasks, double alpha,
                const double *A, const double *B, double *C, double *part, unsigned char *panels) {
  constexpr size_t smem = TcpTile<BN>::kSmem;
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  FNOCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw std::runtime_error("grouped_gemm_tcp: device index out of range");
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
      FNOCC_CUDA(cudaFuncSetAttribute(k_ggemm_tcp<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      done[dev] = true;
    }
  }
  if (pack_blocks > 0x7fffffffLL) throw std::runtime_error("grouped_gemm_tcp: packing grid too large");
  k_tc_pack<BN><<<(unsigned)pack_blocks, kPackThreads, 0, s>>>(tasks, ntasks, A, B, panels);
  FNOCC_CUDA(cudaGetLastError());
  k_ggemm_tcp<BN><<<grid, kTcpThreads, smem, s>>>(tasks, ntasks, alpha, C, part, panels);
}

}  // namespace

// tiles (rows of C x columns of C) of the gathering shapes: 128 x 64,
// 128 x 128, 128 x 256, and the transposed 32 x 128, 64 x 128
void tc_shape(int idx, int *tbm, int *tbn, int *tbk) {
  static const int tm[kGShapesTc] = {kBM, kBM, kBM, 32, 64};
  static const int tn[kGShapesTc] = {64, 128, 256, kBM, kBM};
  if (idx < 0 || idx >= kGShapesTc) throw std::runtime_error("tc_shape: bad shape");
  *tbm = tm[idx];
  *tbn = tn[idx];
  *tbk = kBK;
}

size_t tc_smem_bytes(int idx) {
  switch (idx) {
    case 0: return TcTile<64>::kSmem;
    case 1: return TcTile<128>::kSmem;
    case 2: return TcTile<256>::kSmem;
    case 3: return TcTile<32>::kSmem;
    case 4: return TcTile<64>::kSmem;
    default: throw std::runtime_error("tc_smem_bytes: bad shape");
  }
}

void grouped_gemm_tc(int idx, unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha,
                     const double *A, const double *B, double *C, double *part) {
  switch (idx) {
    case 0: launch_tc<64, false>(grid, s, tasks, ntasks, alpha, A, B, C, part); break;
    case 1: launch_tc<128, false>(grid, s, tasks, ntasks, alpha, A, B, C, part); break;
    case 2: launch_tc<256, false>(grid, s, tasks, ntasks, alpha, A, B, C, part); break;
    case 3: launch_tc<32, true>(grid, s, tasks, ntasks, alpha, A, B, C, part); break;
    case 4: launch_tc<64, true>(grid, s, tasks, ntasks, alpha, A, B, C, part); break;
    default: throw std::runtime_error("grouped_gemm_tc: bad shape");
  }
}

void tcp_block_bytes(int idx, long long *abytes, long long *bbytes) {
  switch (idx) {
    case 0: *abytes = TcpTile<64>::kBlockA; *bbytes = TcpTile<64>::kBlockB; return;
    case 1: *abytes = TcpTile<128>::kBlockA; *bbytes = TcpTile<128>::kBlockB; return;
    case 2: *abytes = TcpTile<256>::kBlockA; *bbytes = TcpTile<256>::kBlockB; return;
    default: throw std::runtime_error("tcp_block_bytes: bad shape");
  }
}

void grouped_gemm_tcp(int idx, unsigned grid, long long pack_blocks, cudaStream_t s, const GTask *tasks, int ntasks,
                      double alpha, const double *A, const double *B, double *C, double *part, unsigned char *panels) {
  switch (idx) {
    case 0: launch_tcp<64>(grid, pack_blocks, s, tasks, ntasks, alpha, A, B, C, part, panels); break;
    case 1: launch_tcp<128>(grid, pack_blocks, s, tasks, ntasks, alpha, A, B, C, part, panels); break;
    case 2: launch_tcp<256>(grid, pack_blocks, s, tasks, ntasks, alpha, A, B, C, part, panels); break;
    default: throw std::runtime_error("grouped_gemm_tcp: bad shape");
  }
}

int tc_status_take(cudaStream_t s) {
  int v = 0;
  FNOCC_CUDA(cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  FNOCC_CUDA(cudaStreamSynchronize(s));
  if (v) {
    const int zero = 0;
    FNOCC_CUDA(cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    FNOCC_CUDA(cudaStreamSynchronize(s));
  }
  return v;
}

}  // namespace fnocc
