/*
 * fnocc.h -- C ABI of libfnocc: frozen-natural-orbital EOM-CCSDT on one GPU.
 *
 * Method: Manisha & Manohar, "Frozen Natural Orbitals based Equation-of-motion
 * coupled-cluster singles, doubles and triples for Ionized, Double-Ionized,
 * Electron Attached and Two-Electron Attached states" (arXiv 2509.14157).
 *   - FNO truncation of the virtual space: Sec. 1.2, Eq. 8-10.
 *   - CCSDT ground state: Eq. 5-7.
 *   - EOM-CCSDT for IP / EA / DIP / DEA: Eq. 1-4.
 *   - XFNO extrapolation over three thresholds: Sec. 2.
 *   - Extensions on the same machinery: the excitation-energy variant EE
 *     (the EOM-CC the four variants build on, Sec. 1), left products and
 *     left eigenvectors, mixed-precision split products, batching of
 *     independent systems and a learned Davidson start.
 *
 * Conventions used by every call:
 *   - Everything is IEEE double, row-major, C-contiguous.
 *   - Spin orbital P = 2*p + s (alpha s = 0, beta s = 1); occupied first.
 *     o = 2*nocc occupied and v = 2*nkept virtual spin orbitals.
 *   - Antisymmetrised integrals <PQ||RS> = <PQ|RS> - <PQ|SR>.
 *   - Packed amplitude layout: unique elements with strictly increasing hole
 *     indices i1<..<i_nh and strictly increasing particle indices
 *     a1<..<a_np, hole tuple major; each tuple list in lexicographic order.
 *     T_n has nh = np = n. EOM components (R1, R2, R3) per variant:
 *       IP  (1,0) (2,1) (3,2)     EA  (0,1) (1,2) (2,3)
 *       DIP (2,0) (3,1) (4,2)     DEA (0,2) (1,3) (2,4)
 *       EE  (1,1) (2,2) (3,3)
 *     An EOM vector is R1, R2, R3 concatenated.
 *   - Operator normalisation: T_n = (1/n!)^2 sum t a^+..i and
 *     R = 1/(nh! np!) sum r a^+..a^+ i..i, i.e. one packed coefficient per
 *     determinant a1^+..a_np^+ i_nh..i1 |Phi_0>.
 *
 * Ownership: host pointers are read (or written) only during the call; the
 * library copies inputs to device memory it owns. A context owns all device
 * memory and frees it in fnocc_destroy. Output buffers belong to the caller.
 *
 * Errors: every call returns an fnocc_status; nothing is thrown across the
 * ABI. fnocc_last_error gives a text for the last failing call on a context.
 * FNOCC_NOT_CONVERGED still fills every output with the last iterate.
 *
 * Fault hook (tests of the error paths; not in the paper): while the
 * environment variable FNOCC_FAULT is set, the library takes one error path
 * on purpose, from the host, without any device fault: "alloc" fails every
 * device allocation above 1 MiB as on a full device (FNOCC_E_NOMEM); "nan"
 * makes ccsdt_solve start from a NaN amplitude (FNOCC_E_NUMERIC at its first
 * energy); "diverge" scales every DIIS extrapolation of the CCSDT amplitudes
 * by 1e3 (FNOCC_E_NUMERIC or FNOCC_NOT_CONVERGED). The variable is read at
 * each use; with it unset the context works normally afterwards.
 *
 * Threading: a context is not thread-safe; use one context per host thread.
 * All GPU work of a context runs on its stream, with eight side streams for
 * the component blocks of the EOM products.
 */
#ifndef FNOCC_H
#define FNOCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FNOCC_OK = 0,
  FNOCC_NOT_CONVERGED = 1,   /* results valid but flagged */
  FNOCC_E_INVALID = -1,      /* bad argument */
  FNOCC_E_NOMEM = -2,        /* device allocation failed */
  FNOCC_E_CUDA = -3,         /* CUDA runtime error */
  FNOCC_E_STATE = -4,        /* call order violated (e.g. ccsdt before a Hamiltonian) */
  FNOCC_E_NUMERIC = -5,      /* NaN or Inf detected */
  FNOCC_E_TIMEOUT = -6       /* a bounded device wait expired */
} fnocc_status;

/* EE: excitation energies (the N-conserving EOM-CCSDT of Sec. 1 that the
 * four particle-number-changing variants build on). */
typedef enum { FNOCC_IP = 0, FNOCC_EA = 1, FNOCC_DIP = 2, FNOCC_DEA = 3, FNOCC_EE = 4 } fnocc_variant;
/* KOOPMANS (recommended): unit vectors on the lowest diagonal entries of the
 * principal block; DIAGONAL: of the whole space (its non-principal unit
 * vectors also carry spin multiplicities the principal block cannot form);
 * LEARNED: principal unit vectors chosen by the context's guess network
 * (fnocc_set_guess_model), which also corrects the preconditioner; KOOPMANS
 * as fallback. Where the chosen block holds fewer elements than guesses are
 * needed, products of the basis (Krylov vectors) fill up, then the
 * lowest-diagonal remaining elements. */
typedef enum { FNOCC_GUESS_KOOPMANS = 0, FNOCC_GUESS_DIAGONAL = 1, FNOCC_GUESS_LEARNED = 2 } fnocc_guess;
typedef enum { FNOCC_CRIT_ABS = 0, FNOCC_CRIT_OCCT = 1 } fnocc_criterion;
/* Arithmetic of the contractions (the single- and double-precision
 * algorithms of Sec. 1). The MIXED kinds run the large contractions as split
 * products on the tensor cores with FP32 accumulation until the residual
 * falls below switch_tol, then refine in FP64: BF16X3 splits each operand
 * (truncated to FP32) into three BF16 slices and sums six slice products
 * (dropped terms below 2^-24 relative); TF32 splits it into two TF32
 * slices and sums three products (about 2^-21 relative). DIIS, Davidson
 * orthogonalisation, the subspace problem and norms are always FP64. */
typedef enum { FNOCC_FP64 = 0, FNOCC_MIXED_BF16X3 = 1, FNOCC_MIXED_TF32 = 2 } fnocc_precision;

typedef struct fnocc_ctx fnocc_ctx;

/* Truncation options (Sec. 1.2; readings of the paper's two unnamed schemes).
 * criterion ABS keeps natural virtuals with occupation >= threshold;
 * OCCT keeps the smallest prefix whose cumulative occupation fraction
 * reaches threshold (e.g. 0.999). nkeep > 0 keeps exactly the top nkeep. */
typedef struct {
  int criterion;        /* fnocc_criterion */
  int nkeep;            /* 0 = use the threshold */
  int scf_maxiter;      /* default 200 */
  double scf_e_tol;     /* default 1e-12 */
  double scf_comm_tol;  /* default 1e-10 */
} fno_options;

typedef struct {
  double e_rhf;           /* reference (RHF) energy */
  double e_mp2;           /* MP2 correlation energy over the full virtual space */
  int nkept;              /* kept spatial virtuals */
  int nvir;               /* all spatial virtuals */
  double kept_fraction;   /* sum kept occupations / sum all occupations */
  int scf_iters;
} fno_info;

typedef struct {
  double tol_res;   /* max |residual| for convergence, default 1e-10 */
  double tol_e;     /* |dE| for convergence, default 1e-12 */
  int maxiter;      /* default 200 */
  int diis;         /* DIIS history length, default 8 (0 = plain Jacobi) */
  int precision;    /* fnocc_precision, default FP64 */
  double switch_tol;/* MIXED: switch to FP64 below this max |residual| (default 1e-6; 0 = never) */
} ccsdt_options;

typedef struct {
  double e_corr;    /* CCSDT correlation energy (Eq. 7) */
  double e_tot;     /* reference + correlation */
  int iters;
  double res_max;   /* max |residual| of the last iteration */
  double seconds;   /* wall time of the solve */
  double seconds_per_iter;
  int iters_mixed;  /* iterations run in MIXED precision */
} ccsdt_info;

typedef struct {
  double tol_res;   /* residual 2-norm per root, default 1e-8 */
  double tol_e;     /* |d omega| per root, default 1e-10 */
  int max_sub;      /* subspace size before a thick restart (keeps the 2*nroots lowest Ritz
                       vectors), default max(6*nroots, nguess+3*nroots) */
  int maxiter;      /* default 200 */
  int nguess;       /* guess vectors, default 2*nroots */
  int precision;    /* fnocc_precision, default FP64 */
  double switch_tol;/* MIXED: FP64 once every residual norm is below this, once the largest
                       residual has not halved for 25 iterations, or after maxiter / 2
                       iterations in mixed precision (default 1e-5; 0 = never); the FP64
                       subspace starts from the Ritz vectors of the chosen roots and of as many
                       further candidates (a thick restart) */
} eom_options;

typedef struct {
  int iters;              /* Davidson iterations */
  int sigma_calls;        /* sigma = H-bar R products evaluated */
  double seconds;
  double seconds_per_iter;
  int complex_roots;      /* roots whose Ritz value had |Im| > 1e-8 */
  double res_max;         /* max residual norm over roots at exit */
  int sigma_calls_mixed;  /* products evaluated in MIXED precision */
  int guess_used;         /* fnocc_guess that produced the roots (LEARNED falls back to DIAGONAL) */
} eom_info;

/* Context ---------------------------------------------------------------- */

/* Creates a context on CUDA device `device`. cuda_stream may be NULL (the
 * context creates its own stream) or a cudaStream_t owned by the caller. */
fnocc_status fnocc_create(fnocc_ctx **ctx, int device, void *cuda_stream);
void fnocc_destroy(fnocc_ctx *ctx);
const char *fnocc_last_error(const fnocc_ctx *ctx);

/* FNO setup (Sec. 1.2, Eq. 8-10) -------------------------------------------
 * h: n*n symmetric one-electron operator; eri: n^4 chemists' (pq|rs) with
 * 8-fold symmetry, in an orthonormal basis (overlap = identity); nocc doubly
 * occupied spatial orbitals. Runs RHF, MP2 amplitudes (Eq. 8-9), the MP2
 * virtual-virtual density (Eq. 10), its eigenvectors (natural orbitals,
 * sorted by occupation), truncation, semicanonicalisation of the kept
 * natural virtuals and the active-space spin-orbital integral transform.
 * occ: optional caller buffer of n - nocc natural occupations (descending),
 * or NULL. The active Hamiltonian stays on the device for the next calls. */
fnocc_status fno_truncate(fnocc_ctx *ctx, const double *h, const double *eri, int n, int nocc,
                          double occ_threshold, const fno_options *opt, fno_info *out,
                          double *occ);

/* Loads an active-space Hamiltonian directly (bypasses fno_truncate): h_mo
 * (n*n) and eri_mo (n^4, chemists' order) are spatial integrals in an
 * orthonormal MO basis whose first nocc orbitals are doubly occupied. f_pq
 * and the reference energy follow from normal ordering. */
fnocc_status fnocc_set_mo_hamiltonian(fnocc_ctx *ctx, const double *h_mo, const double *eri_mo,
                                      int n, int nocc);

/* CCSDT (Eq. 5-7) ------------------------------------------------------------
 * Solves <Phi^n| e^{-T} H e^{T} |Phi_0> = 0, n = 1..3, from T1 = 0,
 * T2 = MP2, T3 = 0 with Jacobi steps and DIIS. opt may be NULL. */
fnocc_status ccsdt_solve(fnocc_ctx *ctx, const ccsdt_options *opt, ccsdt_info *out);

/* One evaluation of the CCSDT residuals and energy for given packed
 * amplitudes (host pointers t1, t2, t3; outputs r1, r2, r3 host, same
 * layout; e_corr the Eq. 7 energy of these amplitudes). */
fnocc_status ccsdt_residual(fnocc_ctx *ctx, const double *t1, const double *t2, const double *t3,
                            double *r1, double *r2, double *r3, double *e_corr);

/* Same with device pointers on the context stream (no host copies). */
fnocc_status ccsdt_residual_dev(fnocc_ctx *ctx, const double *t1, const double *t2,
                                const double *t3, double *r1, double *r2, double *r3,
                                double *e_corr);

/* EOM-CCSDT (Eq. 1-4) ----------------------------------------------------------
 * Lowest nroots roots (by real part) of H-bar in the variant's operator space
 * and target spin sector (IP, EA: 2*dM_s = +1; DIP, DEA, EE: 0), by
 * non-symmetric Davidson. Roots are counted among eigenstates with weight
 * >= 1e-6 in the principal block (1h, 1p, 2h, 2p or 1h1p): the sector also holds
 * states of spin multiplicities the principal block cannot form (quartet
 * 2h1p of IP, quintet 3h1p of DIP, ...), which have no principal weight and
 * which a Davidson started on principal determinants reaches only through
 * rounding; where fewer principal states than nroots exist, the lowest
 * others fill up. Needs a preceding ccsdt_solve (or fnocc_set_amplitudes).
 * energies: total energies E_CC + omega (ascending); omegas may be NULL. */
fnocc_status eom_ccsdt_solve(fnocc_ctx *ctx, int variant, int nroots, int guess,
                             const eom_options *opt, double *energies, double *omegas,
                             eom_info *out);

/* Arithmetic of standalone ccsdt_residual / eom_sigma calls (fnocc_precision;
 * default FP64). The solvers take theirs from their options. */
fnocc_status fnocc_set_precision(fnocc_ctx *ctx, int precision);

/* Tile shape of the grouped contraction kernel (not in the paper; a test
 * and analysis facility of the library). shape -1 (the default) lets the
 * library choose per contraction step (least padded work per busy SM,
 * large FP64 steps timed once and the fastest kept); 0 <= shape < the count
 * returned by fnocc_tile_shape_count forces one shape for every grouped step
 * of the matching arithmetic: shapes below the first mixed-precision shape
 * (the FP64 tiles) apply to FP64 contractions, the others to the split
 * products. Results do not depend on the shape beyond FP64 reassociation.
 * Returns FNOCC_E_INVALID for other values. */
fnocc_status fnocc_set_tile_shape(fnocc_ctx *ctx, int shape);
/* Number of tile shapes (FP64 shapes first, then the split-product shapes);
 * fnocc_tile_shape_first_mixed gives the index of the first split-product
 * shape. */
int fnocc_tile_shape_count(void);
int fnocc_tile_shape_first_mixed(void);
/* Kind of a tile shape: 0 FP64 (CUDA-core FMA tiles), 1 split product on
 * mma.sync (BF16x3, or TF32x3 under FNOCC_MIXED_TF32), 2 BF16x3 split
 * product on the tcgen05 tensor cores with a tensor-memory accumulator,
 * operands gathered by the kernel (128 x 64, 128 x 128, 128 x 256 tiles),
 * 3 the same tiles fed by bulk copies from split BF16 panels that one
 * packing launch per step writes (a panel buffer held by the context, up
 * to 4 GiB per step); kinds 2 and 3 are used by FNOCC_MIXED_BF16X3 only
 * (forcing one under FNOCC_MIXED_TF32 leaves TF32 on its mma.sync tiles);
 * -1 for an index out of range. */
int fnocc_tile_shape_kind(int shape);
/* Process-wide switch of the tile-shape timing (on by default): when on, an
 * FP64 contraction step above 1e8 padded flops times its candidate shapes
 * once and keeps the fastest, so two runs can pick different shapes and
 * their FP64 sums can differ in the last bits (each shape sums in a fixed
 * order). Off: every step runs its estimated shape and repeated runs are
 * bitwise identical. Takes effect for contraction steps issued after the
 * call. */
fnocc_status fnocc_set_autotune(int enable);

/* sigma = (H-bar R)_c for a packed EOM vector (host pointers). R is taken in
 * the variant's target spin sector (2*dM_s = +1 for IP/EA, 0 for DIP/DEA/EE):
 * components outside it do not contribute, and sigma is returned in that
 * sector (zero elsewhere). Likewise every call treats ground-state amplitudes
 * as M_s-conserving. */
fnocc_status eom_sigma(fnocc_ctx *ctx, int variant, const double *r, double *sigma);
fnocc_status eom_sigma_dev(fnocc_ctx *ctx, int variant, const double *r, double *sigma);

/* Launch-sequence replay of the EOM products (not in the paper; a library
 * facility, on by default): once a product's cached R-independent pieces
 * are valid and none of its steps still times tile shapes, its launch
 * sequence is captured in a CUDA graph on the context stream (per variant,
 * direction and arithmetic) and replayed by later products of the same
 * shape, with the input and output copied through two buffers of the
 * vector's size held by the context (vectors above 2^26 elements run
 * without a graph). Results are bitwise those of the plain launches. Off
 * (enable = 0) frees the graphs; per-launch profiling (fnocc_profile)
 * always runs the plain launches. */
fnocc_status fnocc_set_graphs(fnocc_ctx *ctx, int enable);

/* Left product lambda = L^T H-bar, lambda_nu = sum_mu L_mu <mu| (H-bar tau_nu)_c
 * |0> with tau_nu the operator of packed element nu (not in the paper, which
 * names the left vectors L1-L3 only as rate-determining six-index
 * quantities): the transpose of eom_sigma's matrix, same layouts, sector
 * and conventions, evaluated from transposed term lists (fnocc_equation_text
 * kind 2) on the same engine. */
fnocc_status eom_left_sigma(fnocc_ctx *ctx, int variant, const double *l, double *lambda);
fnocc_status eom_left_sigma_dev(fnocc_ctx *ctx, int variant, const double *l, double *lambda);
/* Left eigenvectors: eom_ccsdt_solve with the left product. The eigenvalues
 * are those of the right problem; fnocc_get_block(11..13) then returns the
 * left vectors L1..L3 (unnormalised against the right ones). */
fnocc_status eom_ccsdt_solve_left(fnocc_ctx *ctx, int variant, int nroots, int guess,
                                  const eom_options *opt, double *energies, double *omegas,
                                  eom_info *out);

/* Packed sizes of the three EOM components of a variant for the loaded
 * Hamiltonian (sizes[3]). */
fnocc_status fnocc_eom_sizes(const fnocc_ctx *ctx, int variant, size_t *sizes);

/* Sets packed ground-state amplitudes (host) without solving. */
fnocc_status fnocc_set_amplitudes(fnocc_ctx *ctx, const double *t1, const double *t2,
                                  const double *t3);

/* Dimensions of the loaded Hamiltonian: o, v spin orbitals and the
 * reference energy. */
fnocc_status fnocc_dims(const fnocc_ctx *ctx, int *o, int *v, double *e_ref);

/* Davidson projection: dots[j] = sum_i x[i] * Y[j*ld + i] for j < nvec
 * (device pointers; dots is a device array of nvec doubles), computed with a
 * deterministic two-pass reduction on the context stream; returns after the
 * result is in dots. Scratch for the partial sums comes from the context. */
fnocc_status fnocc_multi_dot(fnocc_ctx *ctx, const double *x, const double *Y, size_t n, size_t ld,
                             int nvec, double *dots);

/* fnocc_multi_dot without any device allocation (the paper has no
 * counterpart; this is a library facility). For callers that cannot allocate
 * device memory: a process whose device memory is owned by another allocator
 * (a framework's caching allocator, a pool sized in advance) must not call
 * cudaMalloc/cudaFree behind its back, and cudaFree synchronises the device.
 * No context is needed; the caller passes the inputs x, Y and the output dots
 * (all device pointers, same meaning as fnocc_multi_dot) and a stream (NULL =
 * the default stream), and the call returns after dots is written.
 * Scratch: a fixed array of 256 x 64 doubles (128 KiB) in the library's own
 * device memory, held on every GPU that loads the library until the process
 * exits. Limit: nvec <= 64; larger nvec (or nvec < 1, n = 0, ld < n, a NULL
 * pointer) returns FNOCC_E_INVALID without touching the GPU.
 * The first call on a device, with that device current, looks up the
 * scratch's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture. Every call waits for its stream
 * (cudaStreamSynchronize) before it returns. A CUDA error already pending on
 * the calling thread when the call starts is left in place for the caller
 * and the call returns FNOCC_E_CUDA without launching anything.
 * Every call shares the one array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The array keeps the last call's partial sums; each call overwrites every
 * element it reads, so nothing needs clearing. */
fnocc_status fnocc_multi_dot_noalloc(const double *x, const double *Y, size_t n, size_t ld, int nvec,
                                     double *dots, void *stream);

/* Copies a packed block to the host. which: 1..3 = T1..T3 of the ground
 * state; 11..13 = R1..R3 of EOM root `root` of the last eom_ccsdt_solve.
 * len must equal the block's packed size. */
fnocc_status fnocc_get_block(fnocc_ctx *ctx, int which, int root, double *buf, size_t len);

/* Batched solves ----------------------------------------------------------
 * Many independent systems (not in the paper; the batching extension): each
 * runs the whole path (fno_truncate, ccsdt_solve, eom_ccsdt_solve for every
 * requested variant) on its own context and CUDA stream, nworkers systems at
 * a time on device `device`, largest first, so that the GPU work of small
 * systems overlaps. omegas[(s * nvariants + k) * nroots + r] receives the
 * ionization / attachment energy omega of root r of variants[k] for system s
 * (total energy = results[s].e_ccsdt + omega); results[s] (optional) its
 * status, energies and timings. Host arrays are read during the call only.
 * Returns FNOCC_OK when every system succeeded, else the first error status
 * met (or FNOCC_NOT_CONVERGED); every system is attempted. */
typedef struct {
  const double *h;       /* n*n, host */
  const double *eri;     /* n^4 chemists' (pq|rs), host */
  int n, nocc;
  double occ_threshold;  /* ABS criterion */
  int nkeep;             /* > 0: keep exactly nkeep natural virtuals */
} fnocc_system;

typedef struct {
  int status;            /* fnocc_status of this system */
  int nkept;
  double e_rhf, e_ccsdt;
  int ccsdt_iters, sigma_calls;
  double seconds;        /* wall time of this system's pipeline */
  char message[128];     /* NUL-terminated text of the first failing call ("" when it succeeded) */
} fnocc_system_result;

fnocc_status fnocc_batch_solve(int device, int nsys, const fnocc_system *systems, int nvariants,
                               const int *variants, int nroots, const ccsdt_options *cc_opt,
                               const eom_options *eom_opt, int nworkers, double *omegas,
                               fnocc_system_result *results);

/* Learned Davidson guess (not in the paper; the learned-guess extension) ----
 * A per-amplitude MLP maps features of each element of the packed operator
 * space to (0) a guess importance, log10 of the element's largest squared
 * amplitude over the lowest roots, and (1) a correction to the diagonal
 * preconditioner, H-bar_mumu - D_mu with D_mu the orbital-energy difference.
 * Network nin = 8 features -> width -> width -> nout = 2, ReLU hidden layers,
 * FP32 parameters (W1 [8 x width], b1, W2 [width x width], b2,
 * W3 [width x 2], b3, row-major, input index first); trained by the
 * library's FP32 kernels (MSE with per-sample per-output weights, Adam),
 * evaluated in BF16 on the tensor cores inside eom_ccsdt_solve. All arrays
 * here are host arrays, row-major [n x 8] / [n x 2]. Training calls on one
 * network must not overlap; solves may share a network (its parameters are
 * only read there). */
typedef struct fnocc_mlp fnocc_mlp;
fnocc_status fnocc_mlp_create(fnocc_mlp **mlp, int device, int nin, int width, int nout, unsigned long long seed);
void fnocc_mlp_destroy(fnocc_mlp *mlp);
const char *fnocc_mlp_last_error(const fnocc_mlp *mlp);
size_t fnocc_mlp_param_count(const fnocc_mlp *mlp);
fnocc_status fnocc_mlp_get_params(fnocc_mlp *mlp, float *params, size_t len);
/* also resets the optimiser state */
fnocc_status fnocc_mlp_set_params(fnocc_mlp *mlp, const float *params, size_t len);
/* y = net(x); bf16 = 1: the BF16 tensor-core inference path, 0: FP32 */
fnocc_status fnocc_mlp_forward(fnocc_mlp *mlp, const float *x, long long n, float *y, int bf16);
/* loss = sum_i sum_o w[i,o] (net(x)[i,o] - t[i,o])^2 / n and its gradient
 * (param_count floats, parameter layout) at the current parameters */
fnocc_status fnocc_mlp_loss_grad(fnocc_mlp *mlp, const float *x, const float *t, const float *w, long long n,
                                 double *loss, float *grad);
/* minibatch Adam (beta 0.9 / 0.999, eps 1e-8), rows shuffled per epoch by a
 * SplitMix64 generator seeded with `seed`; history[epoch] = mean loss (may
 * be NULL). One epoch with batch >= n is exactly one Adam step on loss_grad. */
fnocc_status fnocc_mlp_train(fnocc_mlp *mlp, const float *x, const float *t, const float *w, long long n,
                             int epochs, int batch, float lr, unsigned long long seed, double *history);
/* Parameter file of a network (a trained guess kept for later runs): the
 * 8-byte tag "FNOCCMLP", int32 version (1), nin, width, nout, int64
 * param_count, then the FP32 parameters in the get_params layout, all in the
 * host's byte order. load requires a network of the same shape and resets
 * its optimiser state; a missing, foreign, mismatched or truncated file
 * returns FNOCC_E_INVALID and leaves the parameters unchanged. */
fnocc_status fnocc_mlp_save(fnocc_mlp *mlp, const char *path);
fnocc_status fnocc_mlp_load(fnocc_mlp *mlp, const char *path);

/* Features [dim x 8] of every element of the variant's packed operator space
 * (components concatenated as in eom_sigma): orbital-energy difference D,
 * spin-averaged two-body shift of the element's determinant (sum over hole
 * pairs and particle pairs minus over hole-particle pairs of J_PP for one
 * spatial orbital, J_PQ - K_PQ / 2 otherwise), highest hole and
 * lowest particle energy, mean particle energy, sum over particles of log10
 * of the virtual's natural occupation (0 without FNO), component index,
 * variant. Orbital energies are the diagonal of the active-space Fock
 * operator, integrals the bare antisymmetrised ones. */
fnocc_status fnocc_eom_features(fnocc_ctx *ctx, int variant, float *features);
/* Exact diagonal H-bar_mumu of the sector's elements (others 0), one sigma
 * product per element: training data on small systems. */
fnocc_status fnocc_eom_diagonal(fnocc_ctx *ctx, int variant, double *diag);
/* The same at n chosen elements: out[q] = H-bar_mumu for mu = idx[q] (0 for
 * an element outside the sector), one sigma product per element inside it,
 * so that sampled preconditioner targets on larger training systems cost n
 * products instead of the space's dimension. idx (host, n entries, each in
 * [0, dim)) and out (host, n entries) belong to the caller; n = 0 does
 * nothing. FNOCC_E_INVALID for a bad variant or an index out of range,
 * FNOCC_E_STATE before amplitudes exist. */
fnocc_status fnocc_eom_diagonal_at(fnocc_ctx *ctx, int variant, long long n, const long long *idx, double *out);
/* The network FNOCC_GUESS_LEARNED uses (not owned; NULL detaches). */
fnocc_status fnocc_set_guess_model(fnocc_ctx *ctx, fnocc_mlp *mlp);

/* XFNO (Sec. 2): least-squares line E(f) through (kept_fraction, energy)
 * points evaluated at f = 1 (the paper prints no formula; this is the
 * library's reading). Returns NaN for npts < 1. Pure host function. */
double xfno_extrapolate(const double *kept_fraction, const double *energy, int npts);

/* Same as fno_truncate with h and eri already in device memory (device
 * pointers, read on the context stream). */
fnocc_status fno_truncate_dev(fnocc_ctx *ctx, const double *h_dev, const double *eri_dev, int n,
                              int nocc, double occ_threshold, const fno_options *opt,
                              fno_info *out, double *occ);

/* Text of the term list the library derived for one projected equation
 * (host only, no GPU needed): kind 0 = CCSDT residual of rank out_comp
 * (0 = energy, 1..3), with variant and in_comp ignored; kind 1 = EOM product
 * block sigma_{out_comp} <- R_{in_comp} of `variant` (components 0..2);
 * kind 2 = left product block lambda_{out_comp} <- L_{in_comp}, the
 * transpose of block sigma_{in_comp} <- R_{out_comp} (lambda = L times the
 * product matrix; L enters as the factors r1..r3, not in the paper).
 * Terms are over the T1-similarity-transformed Hamiltonian (f, v) and T2, T3;
 * each line is "coef factor[...] ...", a representative of an orbit of
 * output-index permutations whose full antisymmetriser the caller applies.
 * Writes at most len bytes (NUL-terminated) and returns the full length, or
 * -1 on bad arguments. */
long fnocc_equation_text(int kind, int variant, int out_comp, int in_comp, char *buf, size_t len);

/* Host-only consistency check of the executable plan of the same equation
 * at sizes (o, v) (not in the paper; a test of the library's own
 * bookkeeping): for every grouped contraction step and every tile shape,
 * the launch descriptors must be consistent (CTA ranges tile the grid,
 * tiles match the shape, reduction splits cover K without empty splits in
 * whole K tiles, partial sums and their ordered reduction tile their
 * buffers); for steps with at most max_work multiply-adds the (A, B, C)
 * element offsets the tasks address (flat tables) must also equal, as a
 * multiset, those of the spin-allowed blocks decoded through the per-group
 * offset tables. Returns the number of
 * inconsistencies (0 = consistent) or -1 on bad arguments. No GPU needed. */
long fnocc_plan_selfcheck(int kind, int variant, int out_comp, int in_comp, int o, int v, double max_work);

/* Text of the contraction plan the library builds for the same equation
 * (host only): for every term its GEMM steps with their index groups
 * (packed or not), operands, intermediates and coefficients, planned with
 * the cost model at sizes (o, v); amortize > 0 marks R-independent steps as
 * cached. Same return convention as fnocc_equation_text. */
long fnocc_plan_text(int kind, int variant, int out_comp, int in_comp, int o, int v, double amortize,
                     char *buf, size_t len);

/* Host-only statistics of the executable plan of the same equation at sizes
 * (o, v) (not in the paper; an analysis aid, no GPU needed). stats[10]:
 * [0] grouped FP64 steps run per product (cached R-independent steps
 * excluded), [1] their algorithmic flops, [2] their padded flops at the
 * estimated tile shapes, [3] their model time in seconds on the FP64 pipe
 * (per launch: padded flops x ceil(CTAs / 152) / CTAs at 2 FMA per clock per
 * SM and 2.07 GHz), [4] steps with fewer than 152 CTAs, [5] their flops,
 * [6] other (small-output or GEMV) steps, [7] their flops, [8] doubles of
 * intermediate scratch, [9] doubles of cached R-independent intermediates
 * (device memory of the plan besides its operands). The timed shape
 * of large steps may differ at run time. Returns FNOCC_E_INVALID on bad
 * arguments. */
fnocc_status fnocc_plan_stats(int kind, int variant, int out_comp, int in_comp, int o, int v, double *stats);

/* FP64 throughput of device `device` (not in the paper; the denominators
 * of the FP64 roofline fractions): best of five timed launches of
 * register-only chains of independent FP64 FMAs (fma_tflops) and of FP64
 * tensor-core products mma.sync m8n8k4 (dmma_tflops) on every SM, 2 flops
 * per multiply-add. Needs no context; allocates and frees a small buffer and
 * a stream of its own and takes about a second. */
fnocc_status fnocc_fp64_peak(int device, double *fma_tflops, double *dmma_tflops);

/* Count of kernel launches issued by the context so far. */
uint64_t fnocc_launch_count(const fnocc_ctx *ctx);

/* Algorithmic FP64 flops of the contraction steps run so far (CCSDT residuals
 * and sigma products): sum over planned GEMM steps of 2*M*N*K, where M, N, K
 * count antisymmetry-unique index tuples. */
double fnocc_flop_count(const fnocc_ctx *ctx);

/* Contraction-kernel timing: when enabled, every contraction launch is
 * bracketed by CUDA events on the context stream. Contractions run on one of
 * eight kernel paths: 0 the grouped FP64 gather-GEMM (k_ggemm: all spin blocks
 * of a step in one launch), 1 the same with a split reduction and its
 * ordered sum (k_greduce), 2 the small-output kernel (<= 256 outputs) with
 * its reduction, 3 the row-parallel GEMV, 4 and 5 the grouped BF16
 * three-slice tensor-core kernel (k_ggemm_bf16x3) without / with a split
 * reduction, 6 and 7 the grouped TF32 two-slice kernel (k_ggemm_tf32x3)
 * without / with. fnocc_profile_read returns, for one path (or all with path =
 * -1), the summed device time (ms), the summed algorithmic flops (2*M*N*K)
 * and the number of launches, then resets those counters. */
fnocc_status fnocc_profile(fnocc_ctx *ctx, int enable);
fnocc_status fnocc_profile_read(fnocc_ctx *ctx, int path, double *kernel_ms, double *kernel_flops,
                                uint64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* FNOCC_H */
