// Shared declarations of the fnocc CUDA library: device buffers, index maps
// and the kernel launch wrappers (kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

namespace fnocc {

struct CudaError : std::runtime_error {
  int code;
  CudaError(const std::string &m, int c) : std::runtime_error(m), code(c) {}
};

#define FNOCC_CUDA(x)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess)                                                                    \
      throw ::fnocc::CudaError(std::string(#x) + ": " + cudaGetErrorString(e_), (int)e_);     \
  } while (0)

// Copies outside a context's stream order (plan and constant tables,
// parameter and result reads). A plain cudaMemcpy runs on the legacy default
// stream, which the library's non-blocking streams are not ordered after,
// and from pageable host memory it returns once the data is staged, before
// it has reached the device: a kernel on another stream could then read the
// table before it lands. copy_now goes through the calling thread's default
// stream and copy_after through the stream whose queued work the copy must
// follow; both return with the copy complete.
inline void copy_after(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
  if (!bytes) return;
  FNOCC_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, s));
  FNOCC_CUDA(cudaStreamSynchronize(s));
}
inline void copy_now(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
  copy_after(dst, src, bytes, kind, cudaStreamPerThread);
}

// Host-side fault hook for tests of the error paths (never a device fault):
// while the environment variable FNOCC_FAULT is set, the library takes one
// error path on purpose. "alloc": every device allocation above 1 MiB fails
// as on a full device (FNOCC_E_NOMEM). "nan": ccsdt_solve writes a NaN into
// its first starting amplitude, which only plain arithmetic kernels carry to
// the first energy (FNOCC_E_NUMERIC). "diverge": every DIIS extrapolation of
// the CCSDT amplitudes is scaled by 1e3 (FNOCC_E_NUMERIC or
// FNOCC_NOT_CONVERGED). Read at each use; unset or empty, nothing changes.
enum FaultMode { kFaultNone = 0, kFaultAlloc, kFaultNan, kFaultDiverge };
inline int fault_mode() {
  const char *e = std::getenv("FNOCC_FAULT");
  if (!e || !*e) return kFaultNone;
  if (!std::strcmp(e, "alloc")) return kFaultAlloc;
  if (!std::strcmp(e, "nan")) return kFaultNan;
  if (!std::strcmp(e, "diverge")) return kFaultDiverge;
  return kFaultNone;
}

// Grow-only device buffer owned by a context.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() {}
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void reserve(size_t nbytes) {
    if (nbytes <= bytes && p) return;
    release();
    size_t nb = nbytes ? nbytes : 8;
    if (nb > (size_t(1) << 20) && fault_mode() == kFaultAlloc)
      throw CudaError("cudaMalloc of " + std::to_string(nb) + " bytes failed: injected (FNOCC_FAULT=alloc)",
                      (int)cudaErrorMemoryAllocation);
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
      p = nullptr;
      throw CudaError(std::string("cudaMalloc of ") + std::to_string(nb) + " bytes failed: " +
                          cudaGetErrorString(e), (int)cudaErrorMemoryAllocation);
    }
    bytes = nb;
  }
  double *d() const { return static_cast<double *>(p); }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// Offset map of one GEMM dimension: index m decodes (mixed radix, first group
// most significant) into digits; offset(m) = sum_g tab_g[digit_g].
constexpr int kMaxGroups = 8;
struct DMap {
  int ng = 0;
  long long n[kMaxGroups] = {0};
  const long long *tab[kMaxGroups] = {nullptr};
  long long maxoff = 0;  // host-side bound: sum over groups of the largest table entry
};

// Optional event timing of contraction launches (owned by a context), per
// kernel path: 0 grouped FP64 GEMM, 1 the same with split reduction + ordered
// sum, 2 small-output kernel + reduction, 3 GEMV, 4 / 5 grouped BF16x3 GEMM
// (mma.sync) without / with split reduction, 6 / 7 grouped TF32x3 GEMM
// without / with, 8 / 9 grouped BF16x3 GEMM on tcgen05 without / with,
// 10 / 11 the panel form on tcgen05 (packing launch included) without / with.
constexpr int kGemmPaths = 12;
struct GemmProfile {
  bool enabled = false;
  std::vector<cudaEvent_t> pool;           // events, reused
  std::vector<std::pair<int, int>> pairs;  // (start, stop) indices into pool
  std::vector<double> flops;               // per recorded launch
  std::vector<int> path;                   // per recorded launch
  double ms[kGemmPaths] = {0}, flop_sum[kGemmPaths] = {0};
  uint64_t launches[kGemmPaths] = {0};
  void fold();                             // accumulate completed pairs (synchronises)
};

struct Launch {
  cudaStream_t stream;
  uint64_t *counter;      // incremented per kernel launch
  GemmProfile *prof = nullptr;
  DevBuf *partials = nullptr;  // split-K partial sums (deterministic reduction)
  int precision = 0;  // 0 FP64; tensor-core split products (tiled path): 1 BF16 three-slice, 2 TF32 two-slice
  int sms = 152;       // streaming multiprocessors of the device (grid sizing)
  int force_shape = -1;  // >= 0: every grouped step of the matching arithmetic runs this tile shape
  DevBuf *panels = nullptr;  // split BF16 operand panels of the tcgen05 panel shapes
};

// One sub-GEMM of a grouped launch: C[crow[m] + ccol[n]] += alpha *
// sum_k A[arow[m] + acol[k]] * B[brow[k] + bcol[n]] with flat device offset
// tables (one entry per index). The launch fields (tiles, split, CTA and
// partial offsets) belong to one tile shape.
struct GTask {
  long long M = 0, N = 0, K = 0;
  const long long *arow = nullptr, *acol = nullptr, *brow = nullptr, *bcol = nullptr, *crow = nullptr,
                  *ccol = nullptr;
  long long tiles_n = 0, tiles = 0;  // tiles of the shape, row-major over (m, n) tiles
  long long kchunk = 0;              // reduction length per CTA (multiple of the shape's K tile)
  int ksplit = 1;                    // > 1: partial products to part + part_off, reduced in order
  long long cta_begin = 0;           // first CTA of this task in the grid
  long long part_off = 0;            // doubles, [ksplit][M][N]
  long long red_begin = 0;           // first output of this task in the reduction launch
  int mfast = 0;                     // tcgen05 kernels: tiles ordered with m fastest (consecutive CTAs
                                     // share a column tile of B, the larger operand)
  // tcgen05 panel shapes: split BF16 panels of this task in the panel buffer
  // (bytes), its first block of the packing launch and its 16-wide K steps
  int ksteps = 0;
  long long apanel = 0, bpanel = 0, pk_begin = 0;
};

// A grouped launch: tasks ordered by cta_begin (device array) plus the list
// of tasks with a split reduction.
constexpr int kGShapes = 19;           // FP64 tile shapes (14 with a K tile of 16, 5 of them again with 8)
constexpr int kGShapeBf16 = kGShapes;  // first BF16 three-slice split shape (mixed precision)
constexpr int kGShapesBf16 = 6;        // BF16x3 tiles 64x64, 32x32, 128x16, 16x128, 64x16, 16x64 (mma.sync)
constexpr int kGShapeTc = kGShapeBf16 + kGShapesBf16;  // first tcgen05 BF16x3 shape
constexpr int kGShapesTc = 5;          // tcgen05 BF16x3 tiles 128x64, 128x128, 128x256, and 32x128, 64x128
                                       // computed transposed (TMEM accumulator)
constexpr int kGShapeTcp = kGShapeTc + kGShapesTc;  // first tcgen05 panel shape
constexpr int kGShapesTcp = 3;         // the same tiles fed from split BF16 panels by bulk copies
constexpr int kGShapesAll = kGShapes + kGShapesBf16 + kGShapesTc + kGShapesTcp;
constexpr long long kPanelCapBytes = 1LL << 32;  // split BF16 panels of one step at most (panel tiles)
// kind of a shape: 0 FP64, 1 split product on mma.sync (BF16x3 or TF32x3),
// 2 BF16x3 split product on tcgen05 (operands gathered in the kernel),
// 3 the same from split BF16 panels packed once per step
inline int shape_kind(int shape) {
  return shape < kGShapeBf16 ? 0 : (shape < kGShapeTc ? 1 : (shape < kGShapeTcp ? 2 : 3));
}
// tcgen05 shapes (index 0..kGShapesTc-1): tile, dynamic shared memory,
// launch, and the status word of an expired bounded wait (read and cleared;
// synchronises the stream)
void tc_shape(int idx, int *tbm, int *tbn, int *tbk);
size_t tc_smem_bytes(int idx);
void grouped_gemm_tc(int idx, unsigned grid, cudaStream_t s, const GTask *tasks, int ntasks, double alpha,
                     const double *A, const double *B, double *C, double *part);
int tc_status_take(cudaStream_t s);
// tcgen05 panel shapes (index 0..kGShapesTcp-1): bytes of one 16-wide K step
// of the A (128 rows) and B (BN columns) panels, three BF16 slices each;
// packing launch (one CTA per panel block) and GEMM launch
void tcp_block_bytes(int idx, long long *abytes, long long *bbytes);
void grouped_gemm_tcp(int idx, unsigned grid, long long pack_blocks, cudaStream_t s, const GTask *tasks, int ntasks,
                      double alpha, const double *A, const double *B, double *C, double *part, unsigned char *panels);
struct GroupedLaunch {
  const GTask *tasks = nullptr;
  int ntasks = 0;
  long long ncta = 0;
  const int *split_ids = nullptr;
  int nsplit = 0;
  long long nred = 0, part_need = 0;
  int shape = 0;
  double flops = 0;      // algorithmic flops of the launch (profiling)
  double padded = 0;     // multiply-adds including tile padding x 2
  long long pack_blocks = 0, panel_bytes = 0;  // tcgen05 panel shapes: packing grid and panel buffer
};
// rows, columns and K tile of a shape (FP64 and BF16x3 shapes)
void grouped_shape(int shape, int *tbm, int *tbn, int *tbk);
// runs the launch (and the ordered reduction of split tasks) on L.stream
void grouped_gemm(const Launch &L, const GroupedLaunch &g, double alpha, const double *A, const double *B, double *C);

// C[crow(m) + ccol(n)] (+)= alpha * sum_k A[arow(m)+acol(k)] * B[brow(k)+bcol(n)]
// asize, bsize, csize: element counts of the buffers; every launch checks on
// the host that maxoff(row) + maxoff(col) < size for each operand, so a wrong
// table is reported as an error instead of reaching the device.
// shape: micro-tile of the FP64 tiled path (0..kTileShapes-1), or -1 for the
// shape with the least padding. Returns the shape used (-1 for the GEMV,
// small-output and mixed-precision paths, whose tiles are fixed).
constexpr int kTileShapes = 5;
int gather_gemm(const Launch &L, long long M, long long N, long long K, double alpha,
                const double *A, const DMap &arow, const DMap &acol, const double *B,
                const DMap &brow, const DMap &bcol, double *C, const DMap &crow,
                const DMap &ccol, bool accumulate, long long asize, long long bsize,
                long long csize, int shape = -1);
// C[crow(m)] += alpha * A[arow(m)]
void gather_axpy(const Launch &L, long long M, double alpha, const double *A, const DMap &arow,
                 double *C, const DMap &crow, long long asize, long long csize);

// Antisymmetrise a dense [o^nh v^np] accumulator into packed unique elements:
// out[h,p] = sum_{perm} sign * Y[perm(h), perm(p)] (out overwritten, or
// accumulated into when accumulate). canonical: Y holds every index in the
// canonical order of the engine's tuple tables (beta spin orbitals first,
// then alpha, ascending within each: the engine's accumulators); otherwise
// in spin-orbital order.
void antisym_pack(const Launch &L, const double *Y, int nh, int np, int o, int v,
                  const int *htab, long long nhtup, const int *ptab, long long nptup, double *out,
                  double scale, bool accumulate, bool canonical = true);
// A spin-orbital tensor [n^rank] (rank 1-4, indices occupied first, then
// virtual) rewritten with every index at its canonical position within its
// space, the layout in which the engine reads its operators.
void canonical_layout(const Launch &L, const double *in, int n, int o, int rank, double *out);
// Dense antisymmetric tensor (canonical index order) from packed elements
// (dense zeroed here).
// same result as unpack_dense as one coalesced gather (np >= 1); hrank /
// prank: rank prefix tables of the hole / particle tuple lists
void unpack_dense_rows(const Launch &L, const double *packed, int nh, int np, int o, int v, const long long *hrank,
                       const long long *prank, long long nptup, double *dense);
void unpack_dense(const Launch &L, const double *packed, int nh, int np, int o, int v,
                  const int *htab, long long nhtup, const int *ptab, long long nptup,
                  double *dense);

void fill(const Launch &L, double *x, double val, long long n);
void axpby(const Launch &L, long long n, double a, const double *x, double b, double *y);  // y = a x + b y
void scale_mask(const Launch &L, long long n, double *x, const unsigned char *mask);       // x *= mask
void jacobi_update(const Launch &L, long long n, const double *r, const double *d, double *t);  // t += r/d
void precondition(const Launch &L, long long n, const double *r, const double *d, double theta,
                  const unsigned char *mask, double *out);  // out = mask * r / (theta - d) (mask NULL: 1)
// dst[i] = src[idx[i]] and dst[idx[i]] = src[i] for i < n
void gather_idx(const Launch &L, long long n, const long long *idx, const double *src, double *dst);
void scatter_idx(const Launch &L, long long n, const long long *idx, const double *src, double *dst);
// dots[j] = sum_i x[i] * Y[j*ld + i] for j < nvec  (reduction over i)
void multi_dot(const Launch &L, long long n, const double *x, const double *Y, long long ld,
               int nvec, double *dots_dev, DevBuf &scratch);
// max |x| and sum x^2 into out2[0], out2[1] (NaN reported as an infinite max)
void absmax_sumsq(const Launch &L, long long n, const double *x, double *out2_dev, DevBuf &scratch);
// y (+)= sum_j coef[j] * X[j * ld : j * ld + n], coef_dev: k device doubles
void lincomb(const Launch &L, long long n, const double *X, long long ld, int k, const double *coef_dev, double *y,
             bool accumulate);
// spin-orbital antisymmetrised integrals from spatial (pq|rs) over n spatial orbitals
void spin_orbital_eri(const Launch &L, const double *eri_sp, int n, double *g);
void spin_orbital_h(const Launch &L, const double *h_sp, int n, double *hso);
// f_pq = h_pq + sum_i g[p,i,q,i]; eref2[0] = sum_i h_ii, eref2[1] = 1/2 sum_ij g_ijij
void normal_order(const Launch &L, const double *h, const double *g, int n, int o, double *f,
                  double *eref2_dev);
// L, M matrices of the T1 similarity transformation from t1 [o x v]
void t1_transform_mats(const Launch &L, const double *t1, int o, int v, double *Lm, double *Mm);
// symmetric eigen-decomposition by cyclic Jacobi in one block: A n x n (destroyed),
// evals[n] unsorted, V n x n (columns = eigenvectors). Returns via device flag.
void jacobi_eig(const Launch &L, double *A, int n, double *evals, double *V, int *info_dev);
// out[:, j] = sign_j * in[:, perm[j]] for an n x m column-major-by-index matrix stored row-major
void permute_columns(const Launch &L, const double *in, int rows, int cols_in, const int *perm,
                     int cols_out, double *out);
// fix phase: make the largest |.| entry of each column positive (row-major rows x cols)
void fix_phase(const Launch &L, double *c, int rows, int cols);
// elementwise: out = a + alpha*b + beta*c (any may alias)
void lincomb3(const Launch &L, long long n, double *out, const double *a, double alpha,
              const double *b, double beta, const double *c);
// MP2 amplitudes t[i,j,a,b] = g[a,b,i,j] / (f_ii+f_jj-f_aa-f_bb) over a spin-orbital space
void mp2_amplitudes(const Launch &L, const double *g, const double *fdiag, int n, int o, double *t);
// diagonal of an n x n matrix
void diag_of(const Launch &L, const double *a, int n, double *d);
// dense alpha block of a spin-orbital matrix: out[p,q] = in[2p, 2q]
void alpha_block(const Launch &L, const double *in, int nso, double *out);
// orbital-energy EOM diagonal for packed tuples: d = sum f_pp - sum f_hh
void eom_diag(const Launch &L, const double *fdiag, int o, int nh, int np, const int *htab,
              long long nhtup, const int *ptab, long long nptup, double *d);
// spin-sector mask for packed tuples: 2*M_s change == ms2
void ms_mask(const Launch &L, int nh, int np, const int *htab, long long nhtup, const int *ptab,
             long long nptup, int ms2, unsigned char *mask);
// Jacobi denominators for a packed cluster block (d = sum f_ii - sum f_aa)
void cc_denominators(const Launch &L, const double *fdiag, int o, int rank, const int *htab,
                     long long nhtup, const int *ptab, long long nptup, double *d);

}  // namespace fnocc
