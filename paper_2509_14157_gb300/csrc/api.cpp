// C ABI of libfnocc (include/fnocc.h): context, FNO setup (Sec. 1.2, Eq.
// 8-10), CCSDT (Eq. 5-7), EOM-CCSDT products and Davidson solves (Eq. 1-4)
// for IP / EA / DIP / DEA and the EE and left-vector extensions, XFNO
// (Sec. 2), batching and the learned Davidson start.
#include "../../include/fnocc.h"
#include "mlp.hpp"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "common.hpp"
#include "engine.hpp"
#include "linalg.hpp"
#include "planner.hpp"

using namespace fnocc;

namespace {

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double s() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

struct StatusError : std::runtime_error {
  fnocc_status st;
  StatusError(fnocc_status s, const std::string &m) : std::runtime_error(m), st(s) {}
};

bool valid_precision(int p) { return p == FNOCC_FP64 || p == FNOCC_MIXED_BF16X3 || p == FNOCC_MIXED_TF32; }

DMap stride_map(std::initializer_list<std::pair<long long, long long>> dims, std::vector<long long> &host,
                std::vector<std::pair<DMap *, std::vector<long long>>> &fix, DMap *m) {
  m->ng = (int)dims.size();
  m->maxoff = 0;
  std::vector<long long> offs;
  int g = 0;
  for (auto &d : dims) {
    offs.push_back((long long)host.size());
    for (long long x = 0; x < d.first; ++x) host.push_back(x * d.second);
    m->n[g++] = d.first;
    m->maxoff += (d.first - 1) * d.second;
  }
  fix.push_back({m, offs});
  return *m;
}

// A set of stride maps uploaded once.
struct MapSet {
  std::vector<long long> host;
  std::vector<std::pair<DMap *, std::vector<long long>>> fix;
  DevBuf dev;
  void add(DMap *m, std::initializer_list<std::pair<long long, long long>> dims) { stride_map(dims, host, fix, m); }
  void upload() {
    if (host.empty()) host.push_back(0);
    dev.reserve(host.size() * sizeof(long long));
    copy_now(dev.p, host.data(), host.size() * sizeof(long long), cudaMemcpyHostToDevice);
    for (auto &f : fix)
      for (size_t g = 0; g < f.second.size(); ++g) f.first->tab[g] = dev.as<long long>() + f.second[g];
  }
};

// Maps of one index-transformation pass of a 4-index tensor (dims n_out before
// index `idx`, n_in after), contracting index idx with a (n_in x n_out) matrix.
struct PassMaps {
  DMap arow, acol, brow, bcol, crow, ccol;
};

struct TransformPlan {
  int n_in = 0, n_out = 0;
  PassMaps pass[4];
  PassMaps two[2];  // one-body transform passes (index 0, then index 1)
  MapSet set;
  void build(int ni, int no) {
    n_in = ni;
    n_out = no;
    set.host.clear();
    set.fix.clear();
    for (int idx = 0; idx < 4; ++idx) {
      long long din[4], dout[4];
      for (int k = 0; k < 4; ++k) {
        din[k] = k < idx ? no : ni;
        dout[k] = k <= idx ? no : ni;
      }
      long long sin[4], sout[4];
      sin[3] = sout[3] = 1;
      for (int k = 2; k >= 0; --k) {
        sin[k] = sin[k + 1] * din[k + 1];
        sout[k] = sout[k + 1] * dout[k + 1];
      }
      PassMaps &p = pass[idx];
      set.add(&p.arow, {{no, 1}});
      set.add(&p.acol, {{ni, no}});
      set.add(&p.brow, {{ni, sin[idx]}});
      set.add(&p.crow, {{no, sout[idx]}});
      int others[3], c = 0;
      for (int k = 0; k < 4; ++k)
        if (k != idx) others[c++] = k;
      set.add(&p.bcol, {{din[others[0]], sin[others[0]]}, {din[others[1]], sin[others[1]]}, {din[others[2]], sin[others[2]]}});
      set.add(&p.ccol, {{dout[others[0]], sout[others[0]]}, {dout[others[1]], sout[others[1]]}, {dout[others[2]], sout[others[2]]}});
    }
    // one-body: X[p', q] = sum_p A[p,p'] h[p,q] ; out[p', q'] = sum_q X[p', q] A[q, q']
    set.add(&two[0].arow, {{no, 1}});
    set.add(&two[0].acol, {{ni, no}});
    set.add(&two[0].brow, {{ni, ni}});
    set.add(&two[0].bcol, {{ni, 1}});
    set.add(&two[0].crow, {{no, ni}});
    set.add(&two[0].ccol, {{ni, 1}});
    set.add(&two[1].arow, {{no, 1}});
    set.add(&two[1].acol, {{ni, no}});
    set.add(&two[1].brow, {{ni, 1}});
    set.add(&two[1].bcol, {{no, ni}});
    set.add(&two[1].crow, {{no, 1}});
    set.add(&two[1].ccol, {{no, no}});
    set.upload();
  }
};

// A captured product launch sequence and what it was captured against.
struct ProductGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
  std::vector<uintptr_t> failed;  // key of the last capture that failed
  uint64_t launches = 0;  // kernel launches of one replay
  ProductGraph() {}
  ProductGraph(const ProductGraph &) = delete;
  ProductGraph &operator=(const ProductGraph &) = delete;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key.clear();
  }
  ~ProductGraph() { reset(); }
};

// products of larger spaces are launch-bound no longer and keep their own
// buffers: no graph (and no copies through the fixed buffers)
const size_t kGraphMaxDim = size_t(1) << 26;

// Streams of one EOM product beside the context stream: its nine (output,
// input) component blocks run on nine streams where the two extra
// accumulators per output component take at most kSplitAccBytes, else its
// three output components on three.
constexpr int kSideStreams = 8;
constexpr size_t kSplitAccBytes = size_t(1) << 30;

}  // namespace

struct fnocc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  uint64_t launches = 0;
  GemmProfile prof;
  DevBuf partials;
  double flops_total = 0;
  int precision = 0;          // fnocc_precision of the contractions currently issued
  int default_precision = 0;  // for standalone residual / sigma calls
  int sms = 152;              // multiprocessors of the device (read at creation)
  int force_shape = -1;       // fnocc_set_tile_shape
  DevBuf panels;               // split BF16 operand panels (tcgen05 panel tiles)
  Launch L() { return Launch{stream, &launches, &prof, &partials, precision, sms, force_shape, &panels}; }

  // active Hamiltonian (spin orbitals, bare)
  bool have_ham = false;
  int o = 0, v = 0, n = 0;
  double e_ref = 0;
  DevBuf hso, gso, fso, fdiag;
  std::vector<double> fdiag_host;

  // T1-dressed operators
  DevBuf hd, gd, fdr, tmpA, tmpB, Lm, Mm, tmph, eref2;
  double e_ref_dressed = 0;
  TransformPlan dress_plan;

  TupleTable otab[5], vtab[5];

  // amplitudes: packed [t1 | t2 | t3] in one buffer
  bool have_amps = false;
  size_t nt[4] = {0, 0, 0, 0};
  DevBuf tpk, rpk, t2d, t3d, den;
  double e_corr = 0;

  std::unique_ptr<ExecEquation> cc_eq[4];
  DevBuf Y[4], scratch, red, small, coef;
  // learned guess: the network (not owned), its inference scratch, and the
  // natural occupations of the active virtuals (spatial, semicanonical basis)
  fnocc_mlp *guess_model = nullptr;
  DevBuf mlp_scratch, vocc;
  std::vector<double> virt_occ;

  // EOM
  std::unique_ptr<ExecEquation> eom_eq[kEomVariants][3][3];
  std::unique_ptr<ExecEquation> eom_left_eq[kEomVariants][3][3];  // transposed blocks (left product)
  bool eom_left = false;  // the Davidson applies the left product (eom_ccsdt_solve_left)
  DevBuf rd[3], sy[3];
  uint64_t hbar_version = 0;
  // the dressed operators and dense T2/T3 hold the stored amplitudes' H-bar
  // (cleared by every residual evaluation and by new amplitudes)
  bool hbar_valid = false;
  int plan_o = -1, plan_v = -1;  // shape the contraction plans were built for
  int cache_precision = 0;  // arithmetic of the cached R-independent intermediates
  uint64_t eq_seen[kEomVariants][3][3] = {};  // H-bar version whose cached flops were counted
  uint64_t eq_seen_left[kEomVariants][3][3] = {};
  int last_variant = -1, last_nroots = 0;
  size_t last_dim = 0;
  DevBuf eom_vecs;
  double flops_cc_last = 0, flops_sigma_last = 0;
  // side streams of a product's output components 1 and 2 (component 0 runs
  // on the context stream), each with its own scratch, split partials and
  // panels; fork and join events
  // side streams of the EOM products (their blocks run beside the context
  // stream), with a scratch arena, split-sum partials and tcgen05 panels each
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kSideStreams] = {};
  DevBuf bscratch[kSideStreams], bpartials[kSideStreams], bpanels[kSideStreams];
  DevBuf syx[3][2];  // block-parallel products: accumulators of input components 1 and 2
  // captured product launch sequences [variant][left][precision] and their
  // fixed input / output buffers
  bool use_graphs = true;
  ProductGraph graphs[kEomVariants][2][3];
  DevBuf gx, gs;

  // fno scratch
  DevBuf eri_ao, h_ao, c_mo, dens, fock, jmat, kmat, ctmp, evals, evecs, work, diis_f, diis_e, t2full, w2full,
      dvv, c_act, eri_act, h_act;
  DevBuf ints;  // int scratch
};

namespace {

void set_err(fnocc_ctx *c, const std::string &m) {
  if (c) c->err = m;
}

template <class F>
fnocc_status guarded(fnocc_ctx *c, F &&fn) {
  try {
    return fn();
  } catch (const StatusError &e) {
    set_err(c, e.what());
    return e.st;
  } catch (const CudaError &e) {
    set_err(c, e.what());
    return e.code == (int)cudaErrorMemoryAllocation ? FNOCC_E_NOMEM : FNOCC_E_CUDA;
  } catch (const std::exception &e) {
    set_err(c, e.what());
    return FNOCC_E_INVALID;
  }
}

void sync(fnocc_ctx *c) { FNOCC_CUDA(cudaStreamSynchronize(c->stream)); }

void to_dev(fnocc_ctx *c, DevBuf &b, const double *h, size_t n) {
  b.reserve(n * sizeof(double));
  FNOCC_CUDA(cudaMemcpyAsync(b.p, h, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
}

std::vector<double> to_host(fnocc_ctx *c, const double *d, size_t n) {
  std::vector<double> h(n);
  if (n) FNOCC_CUDA(cudaMemcpyAsync(h.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  sync(c);
  return h;
}

long long ipow(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// (holes, particles) of R1, R2, R3 per variant (IP, EA, DIP, DEA, EE) and the
// sector's 2*M_s change
const int kEom[kEomVariants][3][2] = {{{1, 0}, {2, 1}, {3, 2}}, {{0, 1}, {1, 2}, {2, 3}}, {{2, 0}, {3, 1}, {4, 2}},
                                      {{0, 2}, {1, 3}, {2, 4}}, {{1, 1}, {2, 2}, {3, 3}}};
const int kSectorMs2[kEomVariants] = {1, 1, 0, 0, 0};
// R-independent EOM intermediates are cached per H-bar: the planner charges
// them 1/kSigmaAmortize of their cost (a Davidson solve takes ~100 products);
// one cached intermediate may hold at most 2^28 doubles (2 GiB).
const double kSigmaAmortize = 100.0;
const double kCacheCapDoubles = double(1LL << 28);
// Davidson roots need at least this weight in the principal (1h / 1p / 2h / 2p)
// block: states without it belong to spin multiplicities the principal
// determinants do not reach (see eom_ccsdt_solve)
const double kMinPrincipalWeight = 1e-6;

// ---- Hamiltonian installation ---------------------------------------------------

void install_hamiltonian(fnocc_ctx *c, int nocc, int nact_spatial) {
  // expects c->hso (n x n) and c->gso (n^4) filled for n = 2 * nact_spatial
  c->n = 2 * nact_spatial;
  c->o = 2 * nocc;
  c->v = c->n - c->o;
  Launch L = c->L();
  c->fso.reserve(sizeof(double) * c->n * c->n);
  c->eref2.reserve(sizeof(double) * 2);
  normal_order(L, c->hso.d(), c->gso.d(), c->n, c->o, c->fso.d(), c->eref2.d());
  auto er = to_host(c, c->eref2.d(), 2);
  c->e_ref = er[0] + er[1];
  c->fdiag.reserve(sizeof(double) * c->n);
  diag_of(L, c->fso.d(), c->n, c->fdiag.d());
  c->fdiag_host = to_host(c, c->fdiag.d(), c->n);
  // contraction plans depend on (o, v) only: kept across Hamiltonians of the
  // same shape (their cached intermediates follow the H-bar version)
  if (c->o != c->plan_o || c->v != c->plan_v) {
    for (int k = 0; k <= 4; ++k) {
      c->otab[k].build(c->o, k);
      c->vtab[k].build(c->v, k);
    }
    c->dress_plan.build(c->n, c->n);
    for (int r = 0; r < 4; ++r) c->cc_eq[r].reset();
    for (auto &a : c->eom_eq)
      for (auto &b : a)
        for (auto &e : b) e.reset();
    for (auto &a : c->eom_left_eq)
      for (auto &b : a)
        for (auto &e : b) e.reset();
    c->plan_o = c->o;
    c->plan_v = c->v;
  }
  ++c->hbar_version;
  c->nt[1] = (size_t)binom_ll(c->o, 1) * binom_ll(c->v, 1);
  c->nt[2] = (size_t)binom_ll(c->o, 2) * binom_ll(c->v, 2);
  c->nt[3] = (size_t)binom_ll(c->o, 3) * binom_ll(c->v, 3);
  c->have_ham = true;
  c->have_amps = false;
  c->hbar_valid = false;
  c->last_variant = -1;
}

// ---- T1 similarity transformation -----------------------------------------------

void dress(fnocc_ctx *c, const double *t1) {
  Launch L = c->L();
  L.precision = FNOCC_FP64;  // the T1 transformation and reference energy stay FP64
  const int n = c->n;
  const size_t n4 = (size_t)n * n * n * n;
  c->Lm.reserve(sizeof(double) * n * n);
  c->Mm.reserve(sizeof(double) * n * n);
  c->tmpA.reserve(sizeof(double) * n4);
  c->tmpB.reserve(sizeof(double) * n4);
  c->gd.reserve(sizeof(double) * n4);
  c->hd.reserve(sizeof(double) * n * n);
  c->tmph.reserve(sizeof(double) * n * n);
  c->fdr.reserve(sizeof(double) * n * n);
  t1_transform_mats(L, t1, c->o, c->v, c->Lm.d(), c->Mm.d());
  const TransformPlan &tp = c->dress_plan;
  const double *mats[4] = {c->Lm.d(), c->Lm.d(), c->Mm.d(), c->Mm.d()};
  const double *src = c->gso.d();
  double *dst[4] = {c->tmpA.d(), c->tmpB.d(), c->tmpA.d(), c->gd.d()};
  for (int i = 0; i < 4; ++i) {
    const PassMaps &p = tp.pass[i];
    gather_gemm(L, n, (long long)n * n * n, n, 1.0, mats[i], p.arow, p.acol, src, p.brow, p.bcol, dst[i], p.crow,
                p.ccol, false, (long long)n * n, (long long)n4, (long long)n4);
    src = dst[i];
  }
  gather_gemm(L, n, n, n, 1.0, c->Lm.d(), tp.two[0].arow, tp.two[0].acol, c->hso.d(), tp.two[0].brow,
              tp.two[0].bcol, c->tmph.d(), tp.two[0].crow, tp.two[0].ccol, false, (long long)n * n, (long long)n * n,
              (long long)n * n);
  gather_gemm(L, n, n, n, 1.0, c->Mm.d(), tp.two[1].arow, tp.two[1].acol, c->tmph.d(), tp.two[1].brow,
              tp.two[1].bcol, c->hd.d(), tp.two[1].crow, tp.two[1].ccol, false, (long long)n * n, (long long)n * n,
              (long long)n * n);
  normal_order(L, c->hd.d(), c->gd.d(), n, c->o, c->fdr.d(), c->eref2.d());
  // the contraction engine reads the dressed operators with every index at
  // its canonical position (the order of its tuple tables: one spin block
  // contiguous): rewrite both, swapping buffers with the scratch of the same size
  canonical_layout(L, c->gd.d(), n, c->o, 4, c->tmpA.d());
  std::swap(c->gd.p, c->tmpA.p);
  std::swap(c->gd.bytes, c->tmpA.bytes);
  canonical_layout(L, c->fdr.d(), n, c->o, 2, c->tmph.d());
  std::swap(c->fdr.p, c->tmph.p);
  std::swap(c->fdr.bytes, c->tmph.bytes);
  auto er = to_host(c, c->eref2.d(), 2);
  c->e_ref_dressed = er[0] + er[1];
}

void ensure_cc_plans(fnocc_ctx *c) {
  int rd[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  for (int r = 0; r < 4; ++r)
    if (!c->cc_eq[r]) c->cc_eq[r].reset(new ExecEquation(cc_equation(r), c->o, c->v, rd, 0.0, 0.0, 0, false, c->sms));
}

// residual of packed amplitudes tp (device) into rp (device); returns E_corr
// dense antisymmetric [o^nh v^np] work tensor from packed elements
void unpack(fnocc_ctx *c, const Launch &L, const double *packed, int nh, int np, double *dense) {
  if (np >= 1 && c->v <= 160)
    unpack_dense_rows(L, packed, nh, np, c->o, c->v, c->otab[nh].rank(), c->vtab[np].rank(), c->vtab[np].count,
                      dense);
  else
    unpack_dense(L, packed, nh, np, c->o, c->v, c->otab[nh].dev.as<int>(), c->otab[nh].count,
                 c->vtab[np].dev.as<int>(), c->vtab[np].count, dense);
}

double cc_residual_dev(fnocc_ctx *c, const double *tp, double *rp) {
  c->hbar_valid = false;  // the residual overwrites the dressed operators
  Launch L = c->L();
  ensure_cc_plans(c);
  const int o = c->o, v = c->v;
  const double *t1 = tp, *t2 = tp + c->nt[1], *t3 = tp + c->nt[1] + c->nt[2];
  dress(c, t1);
  c->t2d.reserve(sizeof(double) * ipow(o, 2) * ipow(v, 2));
  c->t3d.reserve(sizeof(double) * std::max<long long>(1, ipow(o, 3) * ipow(v, 3)));
  unpack(c, L, t2, 2, 2, c->t2d.d());
  unpack(c, L, t3, 3, 3, c->t3d.d());
  Operands ops;
  ops.f = c->fdr.d();
  ops.v = c->gd.d();
  ops.t2 = c->t2d.d();
  ops.t3 = c->t3d.d();
  const long long nn = c->n;
  ops.f_size = nn * nn;
  ops.v_size = nn * nn * nn * nn;
  ops.t2_size = ipow(o, 2) * ipow(v, 2);
  ops.t3_size = std::max<long long>(1, ipow(o, 3) * ipow(v, 3));
  // the four residual ranks are independent (each its own equation and
  // accumulator): the triples on the context stream, the energy, singles and
  // doubles on three side streams beside it (per-launch profiling keeps them
  // on the context stream); the arithmetic is the same either way
  const bool fork = !c->prof.enabled;
  struct Join {
    fnocc_ctx *c;
    int n;
    ~Join() {
      for (int i = 0; i < n; ++i)
        if (cudaEventRecord(c->ev_join[i], c->side[i]) == cudaSuccess)
          cudaStreamWaitEvent(c->stream, c->ev_join[i], 0);
    }
  } join{c, 0};
  if (fork) {
    FNOCC_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    for (int i = 0; i < 3; ++i) FNOCC_CUDA(cudaStreamWaitEvent(c->side[i], c->ev_fork, 0));
    join.n = 3;
  }
  double flops = 0;
  size_t offs[4] = {0, 0, c->nt[1], c->nt[1] + c->nt[2]};
  for (int r = 3; r >= 0; --r) {
    Launch Lr = L;
    DevBuf *scr = &c->scratch;
    if (fork && r < 3) {
      Lr.stream = c->side[r];
      Lr.partials = &c->bpartials[r];
      Lr.panels = &c->bpanels[r];
      scr = &c->bscratch[r];
    }
    long long ysz = std::max<long long>(1, ipow(o, r) * ipow(v, r));
    c->Y[r].reserve(sizeof(double) * ysz);
    FNOCC_CUDA(cudaMemsetAsync(c->Y[r].p, 0, sizeof(double) * ysz, Lr.stream));
    c->cc_eq[r]->run(Lr, ops, c->Y[r].d(), ysz, *scr);
    flops += c->cc_eq[r]->flops();
    if (r >= 1)
      antisym_pack(Lr, c->Y[r].d(), r, r, o, v, c->otab[r].dev.as<int>(), c->otab[r].count, c->vtab[r].dev.as<int>(),
                   c->vtab[r].count, rp + offs[r], 1.0, false);
  }
  if (fork) {
    join.n = 0;
    for (int i = 0; i < 3; ++i) {
      FNOCC_CUDA(cudaEventRecord(c->ev_join[i], c->side[i]));
      FNOCC_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join[i], 0));
    }
  }
  c->flops_cc_last = flops;
  c->flops_total += flops;
  if (L.precision == FNOCC_MIXED_BF16X3 && tc_status_take(c->stream))
    throw StatusError(FNOCC_E_TIMEOUT, "a bounded wait of the tcgen05 contraction kernel expired");
  auto y0 = to_host(c, c->Y[0].d(), 1);
  return (c->e_ref_dressed - c->e_ref) + y0[0];
}

void require_ham(fnocc_ctx *c) {
  if (!c->have_ham) throw StatusError(FNOCC_E_STATE, "no Hamiltonian loaded (call fno_truncate or fnocc_set_mo_hamiltonian)");
}

// ---- EOM sigma --------------------------------------------------------------

uint64_t &eq_version(fnocc_ctx *c, int var, int oc, int ic, bool left);

void eom_sizes(const fnocc_ctx *c, int var, size_t *s) {
  for (int k = 0; k < 3; ++k) s[k] = (size_t)binom_ll(c->o, kEom[var][k][0]) * binom_ll(c->v, kEom[var][k][1]);
}

void ensure_eom_plans(fnocc_ctx *c, int var, bool left) {
  int rd[3][2];
  for (int k = 0; k < 3; ++k) {
    rd[k][0] = kEom[var][k][0];
    rd[k][1] = kEom[var][k][1];
  }
  auto &eqs = left ? c->eom_left_eq[var] : c->eom_eq[var];
  for (int oc = 0; oc < 3; ++oc)
    for (int ic = 0; ic < 3; ++ic)
      if (!eqs[oc][ic])
        eqs[oc][ic].reset(new ExecEquation(left ? eom_left_equation(var, oc, ic) : eom_equation(var, oc, ic), c->o,
                                           c->v, rd, kSigmaAmortize, kCacheCapDoubles, kSectorMs2[var], false,
                                           c->sms));
}

// prepares dressed operators and dense T2/T3 from the stored amplitudes
void prepare_hbar(fnocc_ctx *c) {
  if (!c->have_amps) throw StatusError(FNOCC_E_STATE, "no ground-state amplitudes (call ccsdt_solve or fnocc_set_amplitudes)");
  if (c->hbar_valid) return;
  Launch L = c->L();
  const int o = c->o, v = c->v;
  const double *tp = c->tpk.d();
  // the residual accumulators (the T3 one is o^3 v^3 doubles) are dead
  // while products run: their memory goes to the product's work tensors
  for (int r = 0; r < 4; ++r) c->Y[r].release();
  dress(c, tp);
  c->t2d.reserve(sizeof(double) * ipow(o, 2) * ipow(v, 2));
  c->t3d.reserve(sizeof(double) * std::max<long long>(1, ipow(o, 3) * ipow(v, 3)));
  unpack(c, L, tp + c->nt[1], 2, 2, c->t2d.d());
  unpack(c, L, tp + c->nt[1] + c->nt[2], 3, 3, c->t3d.d());
  ++c->hbar_version;
  c->hbar_valid = true;
}

uint64_t &eq_version(fnocc_ctx *c, int var, int oc, int ic, bool left) {
  return left ? c->eq_seen_left[var][oc][ic] : c->eq_seen[var][oc][ic];
}

// the launch sequence of one product: unpack x into the dense work tensors,
// the nine blocks into the dense accumulators, antisymmetrise-pack into s.
// The blocks are independent but for their output: in the block-parallel
// form (small accumulators) block (oc, ic) accumulates into its own tensor
// on its own stream, and the three tensors of an output component are summed
// in input order on the context stream before the pack; otherwise the three
// blocks of an output component share its accumulator and stream. The
// arithmetic (which tensors, which order of the sums) depends only on the
// sizes, so that per-launch profiling, which keeps every launch on the
// context stream (isolated kernel times), gives the same bits.
void sigma_launches(fnocc_ctx *c, int var, const double *x, double *s, bool left, const Launch &L,
                    const Operands &ops) {
  const int o = c->o, v = c->v;
  auto &eqs = left ? c->eom_left_eq[var] : c->eom_eq[var];
  size_t sz[3];
  eom_sizes(c, var, sz);
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    unpack(c, L, x + off, kEom[var][k][0], kEom[var][k][1], c->rd[k].d());
    off += sz[k];
  }
  long long dn[3];
  size_t extra = 0;
  for (int oc = 0; oc < 3; ++oc) {
    dn[oc] = std::max<long long>(1, ipow(o, kEom[var][oc][0]) * ipow(v, kEom[var][oc][1]));
    extra += 2 * sizeof(double) * (size_t)dn[oc];
  }
  const bool split = extra <= kSplitAccBytes;
  if (split)
    for (int oc = 0; oc < 3; ++oc)
      for (int k = 0; k < 2; ++k) c->syx[oc][k].reserve(sizeof(double) * dn[oc]);
  const bool fork = !c->prof.enabled;
  const int nside = fork ? (split ? 8 : 2) : 0;
  struct Join {  // the side streams rejoin the context stream also when a launch throws
    fnocc_ctx *c;
    int n;
    ~Join() {
      for (int i = 0; i < n; ++i)
        if (cudaEventRecord(c->ev_join[i], c->side[i]) == cudaSuccess)
          cudaStreamWaitEvent(c->stream, c->ev_join[i], 0);
    }
  } join{c, 0};
  if (nside > 0) {
    FNOCC_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    for (int i = 0; i < nside; ++i) FNOCC_CUDA(cudaStreamWaitEvent(c->side[i], c->ev_fork, 0));
    join.n = nside;
  }
  off = 0;
  for (int oc = 0; oc < 3; ++oc) {
    const int nh = kEom[var][oc][0], np = kEom[var][oc][1];
    double *Y[3] = {c->sy[oc].d(), split ? c->syx[oc][0].d() : c->sy[oc].d(),
                    split ? c->syx[oc][1].d() : c->sy[oc].d()};
    Launch Lb = L;
    for (int ic = 0; ic < 3; ++ic) {
      const int q = split ? 3 * oc + ic : oc;  // slot: 0 the context stream, q > 0 side stream q - 1
      Lb = L;
      DevBuf *scr = &c->scratch;
      if (q > 0 && q <= nside) {
        Lb.stream = c->side[q - 1];
        Lb.partials = &c->bpartials[q - 1];
        Lb.panels = &c->bpanels[q - 1];
        scr = &c->bscratch[q - 1];
      }
      if (split || ic == 0) FNOCC_CUDA(cudaMemsetAsync(Y[ic], 0, sizeof(double) * dn[oc], Lb.stream));
      eqs[oc][ic]->run(Lb, ops, Y[ic], dn[oc], *scr, c->hbar_version);
    }
    if (!split)  // the component's pack on its own stream, beside the other components
      antisym_pack(Lb, c->sy[oc].d(), nh, np, o, v, c->otab[nh].dev.as<int>(), c->otab[nh].count,
                   c->vtab[np].dev.as<int>(), c->vtab[np].count, s + off, 1.0, false);
    off += sz[oc];
  }
  if (nside > 0) {
    join.n = 0;
    for (int i = 0; i < nside; ++i) {
      FNOCC_CUDA(cudaEventRecord(c->ev_join[i], c->side[i]));
      FNOCC_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join[i], 0));
    }
  }
  if (split) {  // sums in input order and packs on the context stream
    off = 0;
    for (int oc = 0; oc < 3; ++oc) {
      const int nh = kEom[var][oc][0], np = kEom[var][oc][1];
      axpby(L, dn[oc], 1.0, c->syx[oc][0].d(), 1.0, c->sy[oc].d());
      axpby(L, dn[oc], 1.0, c->syx[oc][1].d(), 1.0, c->sy[oc].d());
      antisym_pack(L, c->sy[oc].d(), nh, np, o, v, c->otab[nh].dev.as<int>(), c->otab[nh].count,
                   c->vtab[np].dev.as<int>(), c->vtab[np].count, s + off, 1.0, false);
      off += sz[oc];
    }
  }
}

// everything the captured launches of a product address, and how they were
// chosen: a graph replays only while all of it is unchanged
std::vector<uintptr_t> product_key(fnocc_ctx *c, int var, bool left, const Launch &L, const Operands &ops) {
  auto &eqs = left ? c->eom_left_eq[var] : c->eom_eq[var];
  std::vector<uintptr_t> key = {(uintptr_t)c->hbar_version, (uintptr_t)L.precision, (uintptr_t)(L.force_shape + 1),
                                (uintptr_t)c->gx.p, (uintptr_t)c->gs.p, (uintptr_t)c->scratch.p,
                                (uintptr_t)c->partials.p, (uintptr_t)c->panels.p, (uintptr_t)ops.f,
                                (uintptr_t)ops.v, (uintptr_t)ops.t2, (uintptr_t)ops.t3};
  for (int k = 0; k < 3; ++k) {
    key.push_back((uintptr_t)c->rd[k].p);
    key.push_back((uintptr_t)c->sy[k].p);
  }
  for (int k = 0; k < kSideStreams; ++k) {
    key.push_back((uintptr_t)c->bscratch[k].p);
    key.push_back((uintptr_t)c->bpartials[k].p);
    key.push_back((uintptr_t)c->bpanels[k].p);
  }
  for (int oc = 0; oc < 3; ++oc)
    for (int k = 0; k < 2; ++k) key.push_back((uintptr_t)c->syx[oc][k].p);
  for (int oc = 0; oc < 3; ++oc)
    for (int ic = 0; ic < 3; ++ic) key.push_back((uintptr_t)eqs[oc][ic]->cache_ptr());
  return key;
}

// Captures the product's launch sequence (x and s through the fixed buffers
// gx, gs) into g. Returns false, with nothing captured and nothing launched,
// when the capture fails (a launch error, or another call of this thread
// that a capture does not allow) or when a buffer was reallocated during it,
// whose freed memory the captured launches would address; the caller then
// launches the sequence directly, which reports any error that persists.
bool capture_product(fnocc_ctx *c, int var, bool left, const Launch &L, const Operands &ops,
                     const std::vector<uintptr_t> &key, ProductGraph &g) {
  g.reset();
  const uint64_t l0 = c->launches;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  bool ok = true;
  try {
    sigma_launches(c, var, c->gx.d(), c->gs.d(), left, L, ops);
  } catch (const std::exception &) {
    ok = false;
  }
  const uint64_t launches = c->launches - l0;
  c->launches = l0;
  cudaGraph_t gr = nullptr;
  if (cudaStreamEndCapture(c->stream, &gr) != cudaSuccess) ok = false;
  if (ok && product_key(c, var, left, L, ops) != key) ok = false;
  cudaGraphExec_t ex = nullptr;
  if (ok && gr && cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) {
    ex = nullptr;
    ok = false;
  }
  if (gr) cudaGraphDestroy(gr);
  if (!ok || !ex) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGetLastError();  // a failed capture leaves no error behind
    g.failed = key;
    return false;
  }
  g.exec = ex;
  g.key = key;
  g.launches = launches;
  return true;
}

// s = (H-bar x)_c, or with left = true the left product s = x^T H-bar.
// Once the cached R-independent pieces are valid and no step still times
// its tile shapes, the launch sequence is captured in a CUDA graph (per
// variant, direction and arithmetic) and replayed on later calls, with x
// and s copied through fixed buffers: the few-microsecond launches of the
// small products then run back to back. Per-launch profiling turns it off.
void sigma_dev(fnocc_ctx *c, int var, const double *x, double *s, bool left = false) {
  if (c->precision != c->cache_precision) {  // cached intermediates follow the arithmetic in use
    ++c->hbar_version;
    c->cache_precision = c->precision;
  }
  Launch L = c->L();
  const int o = c->o, v = c->v;
  ensure_eom_plans(c, var, left);
  auto &eqs = left ? c->eom_left_eq[var] : c->eom_eq[var];
  size_t sz[3];
  eom_sizes(c, var, sz);
  const size_t dim = sz[0] + sz[1] + sz[2];
  Operands ops;
  ops.f = c->fdr.d();
  ops.v = c->gd.d();
  ops.t2 = c->t2d.d();
  ops.t3 = c->t3d.d();
  const long long nn = c->n;
  ops.f_size = nn * nn;
  ops.v_size = nn * nn * nn * nn;
  ops.t2_size = ipow(o, 2) * ipow(v, 2);
  ops.t3_size = std::max<long long>(1, ipow(o, 3) * ipow(v, 3));
  for (int k = 0; k < 3; ++k) {
    int nh = kEom[var][k][0], np = kEom[var][k][1];
    long long dn = std::max<long long>(1, ipow(o, nh) * ipow(v, np));
    c->rd[k].reserve(sizeof(double) * dn);
    c->sy[k].reserve(sizeof(double) * dn);
    ops.r[k] = c->rd[k].d();
    ops.r_size[k] = dn;
  }
  double flops = 0;
  bool graph = c->use_graphs && !c->prof.enabled && dim <= kGraphMaxDim;
  for (int oc = 0; oc < 3; ++oc)
    for (int ic = 0; ic < 3; ++ic) {
      ExecEquation &eq = *eqs[oc][ic];
      if (eq.cache_doubles() > 0 && eq_version(c, var, oc, ic, left) != c->hbar_version) flops += eq.cached_flops();
      flops += eq.flops();
      if (eq.needs_refresh(c->hbar_version) || eq.tuning_pending(L)) graph = false;
    }
  if (graph) {
    c->gx.reserve(sizeof(double) * dim);
    c->gs.reserve(sizeof(double) * dim);
    const std::vector<uintptr_t> key = product_key(c, var, left, L, ops);
    ProductGraph &g = c->graphs[var][left ? 1 : 0][L.precision];
    if (!g.exec || g.key != key) {
      // one attempt per key: a capture that failed is not retried until
      // something it depends on changes
      if (g.failed == key || !capture_product(c, var, left, L, ops, key, g)) graph = false;
    }
    if (graph) {
      FNOCC_CUDA(cudaMemcpyAsync(c->gx.p, x, sizeof(double) * dim, cudaMemcpyDeviceToDevice, c->stream));
      FNOCC_CUDA(cudaGraphLaunch(g.exec, c->stream));
      c->launches += g.launches;
      FNOCC_CUDA(cudaMemcpyAsync(s, c->gs.p, sizeof(double) * dim, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  if (!graph) sigma_launches(c, var, x, s, left, L, ops);
  for (int oc = 0; oc < 3; ++oc)
    for (int ic = 0; ic < 3; ++ic) eq_version(c, var, oc, ic, left) = c->hbar_version;
  c->flops_sigma_last = flops;
  c->flops_total += flops;
  if (L.precision == FNOCC_MIXED_BF16X3 && tc_status_take(c->stream))
    throw StatusError(FNOCC_E_TIMEOUT, "a bounded wait of the tcgen05 contraction kernel expired");
}

// ---- small helpers on device vectors ---------------------------------------------

double dot_dev(fnocc_ctx *c, long long n, const double *x, const double *y) {
  c->small.reserve(sizeof(double) * 64);
  multi_dot(c->L(), n, x, y, 0, 1, c->small.d(), c->red);
  return to_host(c, c->small.d(), 1)[0];
}

void absmax_dev(fnocc_ctx *c, long long n, const double *x, double *amax, double *nrm) {
  c->small.reserve(sizeof(double) * 64);
  absmax_sumsq(c->L(), n, x, c->small.d(), c->red);
  auto h = to_host(c, c->small.d(), 2);
  *amax = h[0];
  *nrm = std::sqrt(h[1]);
}

// y = sum_j coef[j] * X[j] (X rows of length n, ld = n)
void combine_rows(fnocc_ctx *c, long long n, const double *X, int k, const std::vector<double> &coef, double *y,
                  bool accumulate) {
  if (k == 0) {
    if (!accumulate) FNOCC_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, c->stream));
    return;
  }
  // coefficients go through their own buffer: stream order keeps them until
  // the launch has read them
  c->coef.reserve(sizeof(double) * std::max<size_t>(64, coef.size()));
  FNOCC_CUDA(cudaMemcpyAsync(c->coef.p, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, c->stream));
  lincomb(c->L(), n, X, n, k, c->coef.d(), y, accumulate);
}

// ---- FNO setup --------------------------------------------------------------------

// symmetric eigen-decomposition of a device n x n matrix; evecs columns sorted
// ascending (descending if desc) with fixed phase; returns eigenvalues (host)
std::vector<double> sym_eig(fnocc_ctx *c, const double *A, int n, double *V, bool desc = false) {
  Launch L = c->L();
  c->work.reserve(sizeof(double) * n * n);
  c->evecs.reserve(sizeof(double) * n * n);
  c->evals.reserve(sizeof(double) * n);
  c->ints.reserve(sizeof(int) * std::max(n, 4));
  FNOCC_CUDA(cudaMemcpyAsync(c->work.p, A, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->stream));
  jacobi_eig(L, c->work.d(), n, c->evals.d(), c->evecs.d(), c->ints.as<int>());
  auto ev = to_host(c, c->evals.d(), n);
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return desc ? ev[a] > ev[b] : ev[a] < ev[b]; });
  FNOCC_CUDA(cudaMemcpyAsync(c->ints.p, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
  permute_columns(L, c->evecs.d(), n, n, c->ints.as<int>(), n, V);
  fix_phase(L, V, n, n);
  sync(c);
  std::vector<double> out(n);
  for (int i = 0; i < n; ++i) out[i] = ev[perm[i]];
  return out;
}

// C = A(rows x k) * B(k x cols), all row-major with leading dims
void matmul(fnocc_ctx *c, int rows, int cols, int k, const double *A, int lda, bool transA, const double *B, int ldb,
            bool transB, double *C, int ldc, long long asz, long long bsz, long long csz) {
  MapSet ms;
  DMap arow, acol, brow, bcol, crow, ccol;
  if (!transA) {
    ms.add(&arow, {{rows, lda}});
    ms.add(&acol, {{k, 1}});
  } else {
    ms.add(&arow, {{rows, 1}});
    ms.add(&acol, {{k, lda}});
  }
  if (!transB) {
    ms.add(&brow, {{k, ldb}});
    ms.add(&bcol, {{cols, 1}});
  } else {
    ms.add(&brow, {{k, 1}});
    ms.add(&bcol, {{cols, ldb}});
  }
  ms.add(&crow, {{rows, ldc}});
  ms.add(&ccol, {{cols, 1}});
  ms.upload();
  gather_gemm(c->L(), rows, cols, k, 1.0, A, arow, acol, B, brow, bcol, C, crow, ccol, false, asz, bsz, csz);
  sync(c);
}

// eri (n_in^4) -> out (n_out^4) with the same n_in x n_out matrix on all indices
void transform4(fnocc_ctx *c, const double *eri, const double *C, int ni, int no, double *out) {
  TransformPlan tp;
  tp.build(ni, no);
  size_t big = (size_t)std::max(ni, no);
  big = big * big * big * big;
  c->tmpA.reserve(sizeof(double) * big);
  c->tmpB.reserve(sizeof(double) * big);
  const double *src = eri;
  double *dst[4] = {c->tmpA.d(), c->tmpB.d(), c->tmpA.d(), out};
  for (int i = 0; i < 4; ++i) {
    long long N = 1;
    for (int k = 0; k < 4; ++k)
      if (k != i) N *= (k < i ? no : ni);
    const PassMaps &p = tp.pass[i];
    long long ssz = ipow(no, i) * ipow(ni, 4 - i), dsz = ipow(no, i + 1) * ipow(ni, 3 - i);
    gather_gemm(c->L(), no, N, ni, 1.0, C, p.arow, p.acol, src, p.brow, p.bcol, dst[i], p.crow, p.ccol, false,
                (long long)ni * no, ssz, dsz);
    src = dst[i];
  }
  sync(c);
}

void transform2(fnocc_ctx *c, const double *h, const double *C, int ni, int no, double *out) {
  // out = C^T h C
  c->tmph.reserve(sizeof(double) * ni * no);
  const long long s1 = (long long)ni * no, s2 = (long long)ni * ni, s3 = (long long)no * no;
  matmul(c, no, ni, ni, C, no, true, h, ni, false, c->tmph.d(), ni, s1, s2, s1);
  matmul(c, no, no, ni, c->tmph.d(), ni, false, C, no, false, out, no, s1, s1, s3);
}

int choose_kept(const std::vector<double> &occ, double thr, int crit, int nkeep) {
  int m = (int)occ.size();
  int k;
  if (nkeep > 0) {
    k = std::min(nkeep, m);
  } else if (crit == FNOCC_CRIT_ABS) {
    k = 0;
    for (double x : occ)
      if (x >= thr) ++k;
  } else {
    double tot = 0;
    for (double x : occ) tot += x;
    if (tot <= 0) {
      k = m;
    } else {
      double cum = 0;
      k = m;
      for (int i = 0; i < m; ++i) {
        cum += occ[i];
        if (cum / tot >= thr - 1e-15) {
          k = i + 1;
          break;
        }
      }
    }
  }
  if (k > 0 && k < m && nkeep <= 0) {
    double tol = 1e-10 * std::max(std::fabs(occ[0]), 1e-300);
    while (k < m && std::fabs(occ[k] - occ[k - 1]) <= tol) ++k;
  }
  return k;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

fnocc_status fnocc_create(fnocc_ctx **out, int device, void *cuda_stream) {
  if (!out) return FNOCC_E_INVALID;
  *out = nullptr;
  fnocc_ctx *c = new (std::nothrow) fnocc_ctx();
  if (!c) return FNOCC_E_NOMEM;
  fnocc_status st = guarded(c, [&]() -> fnocc_status {
    int ndev = 0;
    FNOCC_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) throw StatusError(FNOCC_E_INVALID, "invalid device index");
    FNOCC_CUDA(cudaSetDevice(device));
    c->device = device;
    FNOCC_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
    if (c->sms < 1) c->sms = 1;
    if (cuda_stream) {
      c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      FNOCC_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    for (int i = 0; i < kSideStreams; ++i) {
      FNOCC_CUDA(cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking));
      FNOCC_CUDA(cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming));
    }
    FNOCC_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    return FNOCC_OK;
  });
  if (st != FNOCC_OK) {
    fnocc_destroy(c);
    return st;
  }
  *out = c;
  return FNOCC_OK;
}

void fnocc_destroy(fnocc_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto sd : c->side)
    if (sd) cudaStreamSynchronize(sd);
  bool own = c->own_stream;
  cudaStream_t s = c->stream, side[kSideStreams];
  for (int i = 0; i < kSideStreams; ++i) side[i] = c->side[i];
  for (auto ev : c->prof.pool) cudaEventDestroy(ev);
  for (auto ev : c->ev_join)
    if (ev) cudaEventDestroy(ev);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
  for (auto sd : side)
    if (sd) cudaStreamDestroy(sd);
  if (own && s) cudaStreamDestroy(s);
}

const char *fnocc_last_error(const fnocc_ctx *c) { return c ? c->err.c_str() : "null context"; }

uint64_t fnocc_launch_count(const fnocc_ctx *c) { return c ? c->launches : 0; }

fnocc_status fnocc_set_mo_hamiltonian(fnocc_ctx *c, const double *h_mo, const double *eri_mo, int n, int nocc) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (!h_mo || !eri_mo || n <= 0 || nocc <= 0 || nocc >= n || n > 64)
      throw StatusError(FNOCC_E_INVALID, "invalid Hamiltonian dimensions");
    FNOCC_CUDA(cudaSetDevice(c->device));
    c->virt_occ.clear();
    size_t n4 = (size_t)n * n * n * n;
    to_dev(c, c->h_act, h_mo, (size_t)n * n);
    to_dev(c, c->eri_act, eri_mo, n4);
    int ns = 2 * n;
    c->hso.reserve(sizeof(double) * ns * ns);
    c->gso.reserve(sizeof(double) * (size_t)ns * ns * ns * ns);
    spin_orbital_h(c->L(), c->h_act.d(), n, c->hso.d());
    spin_orbital_eri(c->L(), c->eri_act.d(), n, c->gso.d());
    install_hamiltonian(c, nocc, n);
    sync(c);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_dims(const fnocc_ctx *c, int *o, int *v, double *e_ref) {
  if (!c) return FNOCC_E_INVALID;
  if (!c->have_ham) return FNOCC_E_STATE;
  if (o) *o = c->o;
  if (v) *v = c->v;
  if (e_ref) *e_ref = c->e_ref;
  return FNOCC_OK;
}

static fnocc_status fno_truncate_impl(fnocc_ctx *c, const double *h, const double *eri, bool on_device, int n,
                                      int nocc, double thr, const fno_options *opt, fno_info *out, double *occ_out) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (!h || !eri || n <= 1 || nocc <= 0 || nocc >= n || n > 128) throw StatusError(FNOCC_E_INVALID, "invalid dimensions");
    if (!(thr >= 0.0) || !std::isfinite(thr)) throw StatusError(FNOCC_E_INVALID, "invalid threshold");
    fno_options o;
    o.criterion = FNOCC_CRIT_ABS;
    o.nkeep = 0;
    o.scf_maxiter = 200;
    o.scf_e_tol = 1e-12;
    o.scf_comm_tol = 1e-10;
    if (opt) o = *opt;
    if (o.scf_maxiter <= 0) o.scf_maxiter = 200;
    if (o.scf_e_tol <= 0) o.scf_e_tol = 1e-12;
    if (o.scf_comm_tol <= 0) o.scf_comm_tol = 1e-10;
    if (o.criterion != FNOCC_CRIT_ABS && o.criterion != FNOCC_CRIT_OCCT) throw StatusError(FNOCC_E_INVALID, "bad criterion");
    FNOCC_CUDA(cudaSetDevice(c->device));
    Launch L = c->L();
    const size_t n2 = (size_t)n * n, n4 = n2 * n2;
    if (on_device) {
      c->h_ao.reserve(n2 * sizeof(double));
      c->eri_ao.reserve(n4 * sizeof(double));
      FNOCC_CUDA(cudaMemcpyAsync(c->h_ao.p, h, n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      FNOCC_CUDA(cudaMemcpyAsync(c->eri_ao.p, eri, n4 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      to_dev(c, c->h_ao, h, n2);
      to_dev(c, c->eri_ao, eri, n4);
    }
    c->c_mo.reserve(sizeof(double) * n2);
    c->dens.reserve(sizeof(double) * n2);
    c->fock.reserve(sizeof(double) * n2);
    c->jmat.reserve(sizeof(double) * n2);
    c->kmat.reserve(sizeof(double) * n2);
    c->ctmp.reserve(sizeof(double) * n2);
    const int maxd = 8;
    c->diis_f.reserve(sizeof(double) * n2 * maxd);
    c->diis_e.reserve(sizeof(double) * n2 * maxd);
    // Fock-build maps
    MapSet ms;
    DMap j_arow, j_acol, j_brow, j_bcol, j_crow, j_ccol, k_arow, k_acol, k_brow, k_bcol;
    ms.add(&j_arow, {{(long long)n2, (long long)n2}});
    ms.add(&j_acol, {{(long long)n2, 1}});
    ms.add(&j_brow, {{(long long)n2, 1}});
    ms.add(&j_bcol, {{1, 0}});
    ms.add(&j_crow, {{(long long)n2, 1}});
    ms.add(&j_ccol, {{1, 0}});
    ms.add(&k_arow, {{n, (long long)n2 * n}, {n, n}});
    ms.add(&k_acol, {{n, (long long)n2}, {n, 1}});
    ms.add(&k_brow, {{n, n}, {n, 1}});
    ms.add(&k_bcol, {{1, 0}});
    ms.upload();
    // initial guess: core Hamiltonian
    std::vector<double> eps = sym_eig(c, c->h_ao.d(), n, c->c_mo.d());
    auto build_density = [&]() {
      matmul(c, n, n, nocc, c->c_mo.d(), n, false, c->c_mo.d(), n, true, c->dens.d(), n, (long long)n2, (long long)n2,
             (long long)n2);
    };
    build_density();
    std::vector<double> diis_b(maxd * maxd, 0.0);
    int nd = 0, head = 0;
    double e_old = 0, e = 0;
    int it;
    bool conv = false;
    for (it = 1; it <= o.scf_maxiter; ++it) {
      gather_gemm(L, n2, 1, n2, 1.0, c->eri_ao.d(), j_arow, j_acol, c->dens.d(), j_brow, j_bcol, c->jmat.d(), j_crow,
                  j_ccol, false, (long long)n4, (long long)n2, (long long)n2);
      gather_gemm(L, n2, 1, n2, 1.0, c->eri_ao.d(), k_arow, k_acol, c->dens.d(), k_brow, k_bcol, c->kmat.d(), j_crow,
                  j_ccol, false, (long long)n4, (long long)n2, (long long)n2);
      lincomb3(L, n2, c->fock.d(), c->h_ao.d(), 2.0, c->jmat.d(), -1.0, c->kmat.d());
      lincomb3(L, n2, c->ctmp.d(), c->h_ao.d(), 1.0, c->fock.d(), 0.0, c->fock.d());
      e = dot_dev(c, n2, c->dens.d(), c->ctmp.d());
      // error FD - DF into the DIIS slot
      double *ef = c->diis_e.d() + (size_t)head * n2;
      double *ff = c->diis_f.d() + (size_t)head * n2;
      matmul(c, n, n, n, c->fock.d(), n, false, c->dens.d(), n, false, ef, n, n2, n2, n2);
      matmul(c, n, n, n, c->dens.d(), n, false, c->fock.d(), n, false, c->ctmp.d(), n, n2, n2, n2);
      axpby(L, n2, -1.0, c->ctmp.d(), 1.0, ef);
      FNOCC_CUDA(cudaMemcpyAsync(ff, c->fock.d(), sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
      double emax, enrm;
      absmax_dev(c, n2, ef, &emax, &enrm);
      if (!std::isfinite(e) || !std::isfinite(emax)) throw StatusError(FNOCC_E_NUMERIC, "NaN in SCF");
      if (std::fabs(e - e_old) < o.scf_e_tol && emax < o.scf_comm_tol) {
        conv = true;
        break;
      }
      e_old = e;
      // DIIS bookkeeping (ring buffer of maxd)
      if (nd < maxd) ++nd;
      std::vector<double> dots(maxd);
      c->small.reserve(sizeof(double) * 64);
      multi_dot(L, n2, ef, c->diis_e.d(), n2, nd, c->small.d(), c->red);
      dots = to_host(c, c->small.d(), nd);
      for (int j = 0; j < nd; ++j) {
        diis_b[head * maxd + j] = dots[j];
        diis_b[j * maxd + head] = dots[j];
      }
      head = (head + 1) % maxd;
      double *use = c->fock.d();
      if (nd >= 2) {
        int m = nd;
        std::vector<double> B((m + 1) * (m + 1), 0.0), rhs(m + 1, 0.0), x;
        for (int a = 0; a < m; ++a)
          for (int b = 0; b < m; ++b) B[a * (m + 1) + b] = diis_b[a * maxd + b];
        for (int a = 0; a < m; ++a) B[a * (m + 1) + m] = B[m * (m + 1) + a] = -1.0;
        rhs[m] = -1.0;
        if (solve_linear(m + 1, B, rhs, x)) {
          std::vector<double> coef(x.begin(), x.begin() + m);
          combine_rows(c, n2, c->diis_f.d(), m, coef, c->ctmp.d(), false);
          use = c->ctmp.d();
        }
      }
      eps = sym_eig(c, use, n, c->c_mo.d());
      build_density();
    }
    if (!conv) throw StatusError(FNOCC_E_NUMERIC, "RHF did not converge");
    // canonical orbitals of the converged Fock matrix
    eps = sym_eig(c, c->fock.d(), n, c->c_mo.d());
    const double e_rhf = e;
    const int nvir = n - nocc;
    // MO integrals over the full space
    c->work.reserve(sizeof(double) * n4);
    DevBuf eri_mo;
    eri_mo.reserve(sizeof(double) * n4);
    transform4(c, c->eri_ao.d(), c->c_mo.d(), n, n, eri_mo.d());
    // spin-orbital MP2 amplitudes over the full space (Eq. 8-9)
    const int ns = 2 * n, so = 2 * nocc, sv = 2 * nvir;
    DevBuf gfull, hfull, ffull, fdfull, hmo;
    gfull.reserve(sizeof(double) * (size_t)ns * ns * ns * ns);
    spin_orbital_eri(L, eri_mo.d(), n, gfull.d());
    hmo.reserve(sizeof(double) * n2);
    transform2(c, c->h_ao.d(), c->c_mo.d(), n, n, hmo.d());
    hfull.reserve(sizeof(double) * ns * ns);
    spin_orbital_h(L, hmo.d(), n, hfull.d());
    ffull.reserve(sizeof(double) * ns * ns);
    normal_order(L, hfull.d(), gfull.d(), ns, so, ffull.d(), nullptr);
    fdfull.reserve(sizeof(double) * ns);
    diag_of(L, ffull.d(), ns, fdfull.d());
    size_t t2n = (size_t)so * so * sv * sv;
    c->t2full.reserve(sizeof(double) * std::max<size_t>(t2n, 1));
    mp2_amplitudes(L, gfull.d(), fdfull.d(), ns, so, c->t2full.d());
    // E_MP2 = 1/4 sum <ij||ab> t_ij^ab, <ij||ab> read from gfull through maps
    {
      MapSet em;
      DMap arow, acol, brow, bcol, crow, ccol;
      const long long s3 = (long long)ns * ns * ns, s2 = (long long)ns * ns;
      em.add(&arow, {{1, 0}});
      em.add(&acol, {{so, (long long)so * sv * sv}, {so, (long long)sv * sv}, {sv, sv}, {sv, 1}});
      em.add(&brow, {{so, s3}, {so, s2}, {sv, ns}, {sv, 1}});
      em.add(&bcol, {{1, 0}});
      em.add(&crow, {{1, 0}});
      em.add(&ccol, {{1, 0}});
      em.upload();
      // B must point at g[0,0,o,o] for the (i,j,a,b) -> <ij||ab> block
      c->small.reserve(sizeof(double) * 64);
      const long long gsz = (long long)ns * ns * ns * ns - ((long long)so * ns + so);
      gather_gemm(L, 1, 1, t2n, 0.25, c->t2full.d(), arow, acol, gfull.d() + (size_t)so * ns + so, brow, bcol,
                  c->small.d(), crow, ccol, false, (long long)t2n, gsz, 64);
      sync(c);
    }
    const double e_mp2 = to_host(c, c->small.d(), 1)[0];
    // D_ab = 1/2 sum_ijc t_ij^cb t_ij^ca  (Eq. 10), spin-orbital v x v, then alpha block
    c->dvv.reserve(sizeof(double) * sv * sv);
    {
      MapSet dm;
      DMap arow, acol, brow, bcol, crow, ccol;
      dm.add(&arow, {{sv, 1}});
      dm.add(&acol, {{so, (long long)so * sv * sv}, {so, (long long)sv * sv}, {sv, sv}});
      dm.add(&brow, {{so, (long long)so * sv * sv}, {so, (long long)sv * sv}, {sv, sv}});
      dm.add(&bcol, {{sv, 1}});
      dm.add(&crow, {{sv, sv}});
      dm.add(&ccol, {{sv, 1}});
      dm.upload();
      gather_gemm(L, sv, sv, (long long)so * so * sv, 0.5, c->t2full.d(), arow, acol, c->t2full.d(), brow, bcol,
                  c->dvv.d(), crow, ccol, false, (long long)t2n, (long long)t2n, (long long)sv * sv);
      sync(c);
    }
    DevBuf dsp, uno;
    dsp.reserve(sizeof(double) * nvir * nvir);
    alpha_block(L, c->dvv.d(), sv, dsp.d());
    uno.reserve(sizeof(double) * nvir * nvir);
    std::vector<double> occ = sym_eig(c, dsp.d(), nvir, uno.d(), true);
    int k = choose_kept(occ, thr, o.criterion, o.nkeep);
    double tot = 0, kept = 0;
    for (int i = 0; i < nvir; ++i) {
      tot += occ[i];
      if (i < k) kept += occ[i];
    }
    const double frac = tot > 0 ? kept / tot : 1.0;
    // semicanonicalise: F_vv in the kept NO basis, diagonalised
    int nact = nocc + k;
    std::vector<double> semi_occ;
    c->c_act.reserve(sizeof(double) * n * nact);
    if (k > 0) {
      DevBuf evir, fno_, w, uw, tmp;
      std::vector<double> dg(nvir * nvir, 0.0);
      for (int a = 0; a < nvir; ++a) dg[a * nvir + a] = eps[nocc + a];
      to_dev(c, evir, dg.data(), dg.size());
      tmp.reserve(sizeof(double) * nvir * k);
      fno_.reserve(sizeof(double) * k * k);
      // tmp = diag(eps_v) U_k ; F_no = U_k^T tmp
      DevBuf uk;
      uk.reserve(sizeof(double) * nvir * k);
      FNOCC_CUDA(cudaMemcpy2DAsync(uk.p, sizeof(double) * k, uno.p, sizeof(double) * nvir, sizeof(double) * k, nvir,
                                   cudaMemcpyDeviceToDevice, c->stream));
      const long long nvk = (long long)nvir * k;
      matmul(c, nvir, k, nvir, evir.d(), nvir, false, uk.d(), k, false, tmp.d(), k, (long long)nvir * nvir, nvk, nvk);
      matmul(c, k, k, nvir, uk.d(), k, true, tmp.d(), k, false, fno_.d(), k, nvk, nvk, (long long)k * k);
      w.reserve(sizeof(double) * k * k);
      sym_eig(c, fno_.d(), k, w.d());
      {
        // occupation of each semicanonical virtual: sum_j W[j][a]^2 n_j
        auto wh = to_host(c, w.d(), (size_t)k * k);
        semi_occ.assign(k, 0.0);
        for (int a = 0; a < k; ++a)
          for (int j = 0; j < k; ++j) semi_occ[a] += wh[(size_t)j * k + a] * wh[(size_t)j * k + a] * occ[j];
      }
      uw.reserve(sizeof(double) * nvir * k);
      matmul(c, nvir, k, k, uk.d(), k, false, w.d(), k, false, uw.d(), k, nvk, (long long)k * k, nvk);
      // C_vir_new = C[:, nocc:] * UW
      DevBuf cv;
      cv.reserve(sizeof(double) * n * k);
      matmul(c, n, k, nvir, c->c_mo.d() + nocc, n, false, uw.d(), k, false, cv.d(), k, (long long)n2 - nocc, nvk,
             (long long)n * k);
      fix_phase(L, cv.d(), n, k);
      FNOCC_CUDA(cudaMemcpy2DAsync(c->c_act.d() + nocc, sizeof(double) * nact, cv.p, sizeof(double) * k,
                                   sizeof(double) * k, n, cudaMemcpyDeviceToDevice, c->stream));
      sync(c);
    }
    FNOCC_CUDA(cudaMemcpy2DAsync(c->c_act.p, sizeof(double) * nact, c->c_mo.p, sizeof(double) * n,
                                 sizeof(double) * nocc, n, cudaMemcpyDeviceToDevice, c->stream));
    // active-space integrals
    c->eri_act.reserve(sizeof(double) * (size_t)nact * nact * nact * nact);
    transform4(c, c->eri_ao.d(), c->c_act.d(), n, nact, c->eri_act.d());
    c->h_act.reserve(sizeof(double) * nact * nact);
    transform2(c, c->h_ao.d(), c->c_act.d(), n, nact, c->h_act.d());
    const int nsa = 2 * nact;
    c->hso.reserve(sizeof(double) * nsa * nsa);
    c->gso.reserve(sizeof(double) * (size_t)nsa * nsa * nsa * nsa);
    spin_orbital_h(L, c->h_act.d(), nact, c->hso.d());
    spin_orbital_eri(L, c->eri_act.d(), nact, c->gso.d());
    install_hamiltonian(c, nocc, nact);
    c->virt_occ = semi_occ;
    sync(c);
    if (out) {
      out->e_rhf = e_rhf;
      out->e_mp2 = e_mp2;
      out->nkept = k;
      out->nvir = nvir;
      out->kept_fraction = frac;
      out->scf_iters = it;
    }
    if (occ_out) std::memcpy(occ_out, occ.data(), sizeof(double) * nvir);
    return FNOCC_OK;
  });
}

fnocc_status fno_truncate(fnocc_ctx *c, const double *h, const double *eri, int n, int nocc, double thr,
                          const fno_options *opt, fno_info *out, double *occ_out) {
  return fno_truncate_impl(c, h, eri, false, n, nocc, thr, opt, out, occ_out);
}

fnocc_status fno_truncate_dev(fnocc_ctx *c, const double *h, const double *eri, int n, int nocc, double thr,
                              const fno_options *opt, fno_info *out, double *occ_out) {
  return fno_truncate_impl(c, h, eri, true, n, nocc, thr, opt, out, occ_out);
}

double fnocc_flop_count(const fnocc_ctx *c) { return c ? c->flops_total : 0.0; }

fnocc_status fnocc_profile(fnocc_ctx *c, int enable) {
  if (!c) return FNOCC_E_INVALID;
  c->prof.enabled = enable != 0;
  return FNOCC_OK;
}

fnocc_status fnocc_profile_read(fnocc_ctx *c, int path, double *ms, double *flops, uint64_t *launches) {
  if (!c || path < -1 || path >= kGemmPaths) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    GemmProfile &pr = c->prof;
    FNOCC_CUDA(cudaStreamSynchronize(c->stream));
    pr.fold();
    double m = 0, f = 0;
    uint64_t n = 0;
    for (int k = 0; k < kGemmPaths; ++k)
      if (path < 0 || path == k) {
        m += pr.ms[k];
        f += pr.flop_sum[k];
        n += pr.launches[k];
      }
    if (ms) *ms = m;
    if (flops) *flops = f;
    if (launches) *launches = n;
    for (int k = 0; k < kGemmPaths; ++k)
      if (path < 0 || path == k) {
        pr.ms[k] = 0;
        pr.flop_sum[k] = 0;
        pr.launches[k] = 0;
      }
    return FNOCC_OK;
  });
}

fnocc_status fnocc_set_amplitudes(fnocc_ctx *c, const double *t1, const double *t2, const double *t3) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    require_ham(c);
    if (!t1 || !t2 || (!t3 && c->nt[3] > 0)) throw StatusError(FNOCC_E_INVALID, "null amplitude pointer");
    size_t tot = c->nt[1] + c->nt[2] + c->nt[3];
    c->tpk.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    FNOCC_CUDA(cudaMemcpyAsync(c->tpk.d(), t1, sizeof(double) * c->nt[1], cudaMemcpyHostToDevice, c->stream));
    FNOCC_CUDA(cudaMemcpyAsync(c->tpk.d() + c->nt[1], t2, sizeof(double) * c->nt[2], cudaMemcpyHostToDevice, c->stream));
    if (c->nt[3])
      FNOCC_CUDA(cudaMemcpyAsync(c->tpk.d() + c->nt[1] + c->nt[2], t3, sizeof(double) * c->nt[3], cudaMemcpyHostToDevice,
                                 c->stream));
    sync(c);
    c->have_amps = true;
    c->rpk.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    c->e_corr = cc_residual_dev(c, c->tpk.d(), c->rpk.d());
    return FNOCC_OK;
  });
}

fnocc_status ccsdt_residual_dev(fnocc_ctx *c, const double *t1, const double *t2, const double *t3, double *r1,
                                double *r2, double *r3, double *e_corr) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    require_ham(c);
    FNOCC_CUDA(cudaSetDevice(c->device));
    size_t tot = c->nt[1] + c->nt[2] + c->nt[3];
    c->tpk.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    c->rpk.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    auto cp = [&](double *dst, const double *src, size_t n) {
      if (n) FNOCC_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    };
    DevBuf tin;
    tin.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    cp(tin.d(), t1, c->nt[1]);
    cp(tin.d() + c->nt[1], t2, c->nt[2]);
    cp(tin.d() + c->nt[1] + c->nt[2], t3, c->nt[3]);
    c->precision = c->default_precision;
    double e = cc_residual_dev(c, tin.d(), c->rpk.d());
    c->precision = FNOCC_FP64;
    cp(r1, c->rpk.d(), c->nt[1]);
    cp(r2, c->rpk.d() + c->nt[1], c->nt[2]);
    cp(r3, c->rpk.d() + c->nt[1] + c->nt[2], c->nt[3]);
    sync(c);
    if (e_corr) *e_corr = e;
    return FNOCC_OK;
  });
}

fnocc_status ccsdt_residual(fnocc_ctx *c, const double *t1, const double *t2, const double *t3, double *r1, double *r2,
                            double *r3, double *e_corr) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    require_ham(c);
    if (!t1 || !t2 || !r1 || !r2 || (c->nt[3] && (!t3 || !r3))) throw StatusError(FNOCC_E_INVALID, "null pointer");
    FNOCC_CUDA(cudaSetDevice(c->device));
    size_t tot = c->nt[1] + c->nt[2] + c->nt[3];
    DevBuf tin, rout;
    tin.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    rout.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    FNOCC_CUDA(cudaMemcpyAsync(tin.d(), t1, sizeof(double) * c->nt[1], cudaMemcpyHostToDevice, c->stream));
    FNOCC_CUDA(cudaMemcpyAsync(tin.d() + c->nt[1], t2, sizeof(double) * c->nt[2], cudaMemcpyHostToDevice, c->stream));
    if (c->nt[3])
      FNOCC_CUDA(cudaMemcpyAsync(tin.d() + c->nt[1] + c->nt[2], t3, sizeof(double) * c->nt[3], cudaMemcpyHostToDevice,
                                 c->stream));
    c->precision = c->default_precision;
    double e = cc_residual_dev(c, tin.d(), rout.d());
    c->precision = FNOCC_FP64;
    FNOCC_CUDA(cudaMemcpyAsync(r1, rout.d(), sizeof(double) * c->nt[1], cudaMemcpyDeviceToHost, c->stream));
    FNOCC_CUDA(cudaMemcpyAsync(r2, rout.d() + c->nt[1], sizeof(double) * c->nt[2], cudaMemcpyDeviceToHost, c->stream));
    if (c->nt[3])
      FNOCC_CUDA(cudaMemcpyAsync(r3, rout.d() + c->nt[1] + c->nt[2], sizeof(double) * c->nt[3], cudaMemcpyDeviceToHost,
                                 c->stream));
    sync(c);
    if (e_corr) *e_corr = e;
    return FNOCC_OK;
  });
}

fnocc_status ccsdt_solve(fnocc_ctx *c, const ccsdt_options *opt, ccsdt_info *out) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    require_ham(c);
    FNOCC_CUDA(cudaSetDevice(c->device));
    Timer timer;
    ccsdt_options o{1e-10, 1e-12, 200, 8, FNOCC_FP64, 1e-6};
    if (opt) o = *opt;
    if (!valid_precision(o.precision))
      throw StatusError(FNOCC_E_INVALID, "bad precision");
    if (o.switch_tol < 0) o.switch_tol = 0;
    struct PrecisionGuard {
      fnocc_ctx *c;
      ~PrecisionGuard() { c->precision = FNOCC_FP64; }
    } guard{c};
    c->precision = o.precision;
    int iters_mixed = 0;
    if (o.tol_res <= 0) o.tol_res = 1e-10;
    if (o.tol_e <= 0) o.tol_e = 1e-12;
    if (o.maxiter <= 0) o.maxiter = 200;
    if (o.diis < 0) o.diis = 0;
    if (o.diis > 16) o.diis = 16;
    Launch L = c->L();
    const int oo = c->o, vv = c->v;
    const size_t n1 = c->nt[1], n2 = c->nt[2], n3 = c->nt[3], tot = n1 + n2 + n3;
    c->tpk.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    c->rpk.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    c->den.reserve(sizeof(double) * std::max<size_t>(tot, 1));
    // denominators
    for (int r = 1; r <= 3; ++r) {
      size_t off = (r >= 2 ? n1 : 0) + (r >= 3 ? n2 : 0);
      cc_denominators(L, c->fdiag.d(), oo, r, c->otab[r].dev.as<int>(), c->otab[r].count, c->vtab[r].dev.as<int>(),
                      c->vtab[r].count, c->den.d() + off);
    }
    // T1 = 0, T2 = MP2 (packed), T3 = 0
    FNOCC_CUDA(cudaMemsetAsync(c->tpk.p, 0, sizeof(double) * tot, c->stream));
    {
      DevBuf t2dense;
      t2dense.reserve(sizeof(double) * (size_t)oo * oo * vv * vv);
      mp2_amplitudes(L, c->gso.d(), c->fdiag.d(), c->n, oo, t2dense.d());
      antisym_pack(L, t2dense.d(), 2, 2, oo, vv, c->otab[2].dev.as<int>(), c->otab[2].count, c->vtab[2].dev.as<int>(),
                   c->vtab[2].count, c->tpk.d() + n1, 0.25, false, false);  // MP2 amplitudes in spin-orbital order
      sync(c);
    }
    if (fault_mode() == kFaultNan) {  // test hook: a poisoned starting amplitude
      const double bad = std::nan("");
      copy_after(c->tpk.p, &bad, sizeof(double), cudaMemcpyHostToDevice, c->stream);
    }
    const int md = o.diis;
    DevBuf hv, he;
    if (md > 0) {
      hv.reserve(sizeof(double) * tot * md);
      he.reserve(sizeof(double) * tot * md);
    }
    std::vector<double> bmat(md * md, 0.0);
    int nd = 0, head = 0;
    double e_old = 0, e = 0, rmax = 0, rn = 0;
    bool conv = false;
    int it;
    for (it = 1; it <= o.maxiter; ++it) {
      if (c->precision != FNOCC_FP64) ++iters_mixed;
      e = cc_residual_dev(c, c->tpk.d(), c->rpk.d());
      absmax_dev(c, tot, c->rpk.d(), &rmax, &rn);
      if (!std::isfinite(e) || !std::isfinite(rmax)) throw StatusError(FNOCC_E_NUMERIC, "NaN/Inf in CCSDT iterations");
      if (c->precision != FNOCC_FP64 && o.switch_tol > 0 && rmax < o.switch_tol) {
        // refinement: from here on every contraction is FP64; the iterate is kept
        c->precision = FNOCC_FP64;
        e_old = e;
        continue;
      }
      if (it > 1 && rmax < o.tol_res && std::fabs(e - e_old) < o.tol_e) {
        conv = true;
        break;
      }
      e_old = e;
      // Jacobi step, error = R / D
      jacobi_update(L, tot, c->rpk.d(), c->den.d(), c->tpk.d());
      if (md > 0) {
        double *ev = he.d() + (size_t)head * tot;
        double *tv = hv.d() + (size_t)head * tot;
        FNOCC_CUDA(cudaMemsetAsync(ev, 0, sizeof(double) * tot, c->stream));
        jacobi_update(L, tot, c->rpk.d(), c->den.d(), ev);
        FNOCC_CUDA(cudaMemcpyAsync(tv, c->tpk.d(), sizeof(double) * tot, cudaMemcpyDeviceToDevice, c->stream));
        if (nd < md) ++nd;
        c->small.reserve(sizeof(double) * 64);
        multi_dot(L, tot, ev, he.d(), tot, nd, c->small.d(), c->red);
        auto dots = to_host(c, c->small.d(), nd);
        for (int j = 0; j < nd; ++j) {
          bmat[head * md + j] = dots[j];
          bmat[j * md + head] = dots[j];
        }
        head = (head + 1) % md;
        if (nd >= 2) {
          int m = nd;
          std::vector<double> B((m + 1) * (m + 1), 0.0), rhs(m + 1, 0.0), x;
          for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) B[a * (m + 1) + b] = bmat[a * md + b];
          for (int a = 0; a < m; ++a) B[a * (m + 1) + m] = B[m * (m + 1) + a] = -1.0;
          rhs[m] = -1.0;
          if (solve_linear(m + 1, B, rhs, x)) {
            std::vector<double> coef(x.begin(), x.begin() + m);
            if (fault_mode() == kFaultDiverge)  // test hook: a corrupted extrapolation
              for (double &cf : coef) cf *= 1e3;
            combine_rows(c, tot, hv.d(), m, coef, c->tpk.d(), false);
          }
        }
      }
    }
    c->have_amps = true;
    c->e_corr = e;
    double secs = timer.s();
    if (out) {
      out->e_corr = e;
      out->e_tot = c->e_ref + e;
      out->iters = conv ? it : o.maxiter;
      out->res_max = rmax;
      out->seconds = secs;
      out->seconds_per_iter = secs / std::max(1, conv ? it : o.maxiter);
      out->iters_mixed = iters_mixed;
    }
    return conv ? FNOCC_OK : FNOCC_NOT_CONVERGED;
  });
}

fnocc_status fnocc_set_precision(fnocc_ctx *c, int precision) {
  if (!c || (!valid_precision(precision))) return FNOCC_E_INVALID;
  c->default_precision = precision;
  return FNOCC_OK;
}

fnocc_status fnocc_set_tile_shape(fnocc_ctx *c, int shape) {
  if (!c || shape < -1 || shape >= fnocc_tile_shape_count()) return FNOCC_E_INVALID;
  c->force_shape = shape;
  return FNOCC_OK;
}

int fnocc_tile_shape_count(void) { return kGShapesAll; }

fnocc_status fnocc_set_graphs(fnocc_ctx *c, int enable) {
  if (!c) return FNOCC_E_INVALID;
  c->use_graphs = enable != 0;
  if (!c->use_graphs)
    for (auto &a : c->graphs)
      for (auto &b : a)
        for (auto &g : b) g.reset();
  return FNOCC_OK;
}

fnocc_status fnocc_set_autotune(int enable) {
  ExecEquation::autotune = enable != 0;
  return FNOCC_OK;
}
int fnocc_tile_shape_first_mixed(void) { return kGShapeBf16; }
int fnocc_tile_shape_kind(int shape) { return shape < 0 || shape >= kGShapesAll ? -1 : shape_kind(shape); }

fnocc_status fnocc_eom_sizes(const fnocc_ctx *c, int variant, size_t *sizes) {
  if (!c || !sizes || variant < 0 || variant >= kEomVariants) return FNOCC_E_INVALID;
  if (!c->have_ham) return FNOCC_E_STATE;
  eom_sizes(c, variant, sizes);
  return FNOCC_OK;
}


namespace {

fnocc_status product_dev(fnocc_ctx *c, int variant, const double *r, double *s, bool left) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (variant < 0 || variant >= kEomVariants) throw StatusError(FNOCC_E_INVALID, "bad variant");
    require_ham(c);
    FNOCC_CUDA(cudaSetDevice(c->device));
    prepare_hbar(c);
    c->precision = c->default_precision;
    sigma_dev(c, variant, r, s, left);
    c->precision = FNOCC_FP64;
    sync(c);
    return FNOCC_OK;
  });
}

fnocc_status product_host(fnocc_ctx *c, int variant, const double *r, double *s, bool left) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (variant < 0 || variant >= kEomVariants || !r || !s) throw StatusError(FNOCC_E_INVALID, "bad argument");
    require_ham(c);
    FNOCC_CUDA(cudaSetDevice(c->device));
    size_t sz[3];
    eom_sizes(c, variant, sz);
    size_t dim = sz[0] + sz[1] + sz[2];
    DevBuf x, y;
    x.reserve(sizeof(double) * dim);
    y.reserve(sizeof(double) * dim);
    FNOCC_CUDA(cudaMemcpyAsync(x.p, r, sizeof(double) * dim, cudaMemcpyHostToDevice, c->stream));
    prepare_hbar(c);
    c->precision = c->default_precision;
    sigma_dev(c, variant, x.d(), y.d(), left);
    c->precision = FNOCC_FP64;
    FNOCC_CUDA(cudaMemcpyAsync(s, y.p, sizeof(double) * dim, cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    return FNOCC_OK;
  });
}

}  // namespace

fnocc_status eom_sigma(fnocc_ctx *c, int variant, const double *r, double *s) {
  return product_host(c, variant, r, s, false);
}

fnocc_status eom_sigma_dev(fnocc_ctx *c, int variant, const double *r, double *s) {
  return product_dev(c, variant, r, s, false);
}

fnocc_status eom_left_sigma(fnocc_ctx *c, int variant, const double *l, double *lambda) {
  return product_host(c, variant, l, lambda, true);
}

fnocc_status eom_left_sigma_dev(fnocc_ctx *c, int variant, const double *l, double *lambda) {
  return product_dev(c, variant, l, lambda, true);
}

// features [dim x kMlpFeatures] of the variant's operator space (device)
void eom_features_dev(fnocc_ctx *c, int variant, float *out) {
  const int o = c->o, v = c->v;
  std::vector<float> vl(std::max(v, 1), 0.f);
  if (!c->virt_occ.empty())
    for (int a = 0; a < v; ++a) vl[a] = (float)std::log10(std::max(c->virt_occ[a / 2], 1e-12));
  c->vocc.reserve(sizeof(float) * vl.size());
  FNOCC_CUDA(cudaMemcpyAsync(c->vocc.p, vl.data(), sizeof(float) * vl.size(), cudaMemcpyHostToDevice, c->stream));
  size_t sz[3];
  eom_sizes(c, variant, sz);
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    const int nh = kEom[variant][k][0], np = kEom[variant][k][1];
    eom_features(c->stream, nh, np, o, c->n, c->otab[nh].dev.as<int>(), c->otab[nh].count,
                 c->vtab[np].dev.as<int>(), c->vtab[np].count, c->fdiag.d(), c->gso.d(), c->vocc.as<float>(), k,
                 variant, out + off * kMlpFeatures);
    off += sz[k];
  }
}

fnocc_status eom_solve_once(fnocc_ctx *c, int variant, int nroots, int guess, const eom_options *opt,
                            double *energies, double *omegas, eom_info *out) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (variant < 0 || variant >= kEomVariants) throw StatusError(FNOCC_E_INVALID, "bad variant");
    if (nroots <= 0 || !energies) throw StatusError(FNOCC_E_INVALID, "bad nroots or null energies");
    if (guess != FNOCC_GUESS_KOOPMANS && guess != FNOCC_GUESS_DIAGONAL && guess != FNOCC_GUESS_LEARNED)
      throw StatusError(FNOCC_E_INVALID, "bad guess");
    if (guess == FNOCC_GUESS_LEARNED && (!c->guess_model || !c->guess_model->net))
      throw StatusError(FNOCC_E_STATE, "no guess network (fnocc_set_guess_model)");
    require_ham(c);
    FNOCC_CUDA(cudaSetDevice(c->device));
    Timer timer;
    eom_options o{1e-8, 1e-10, 0, 200, 0, FNOCC_FP64, 1e-5};
    if (opt) o = *opt;
    if (!valid_precision(o.precision))
      throw StatusError(FNOCC_E_INVALID, "bad precision");
    if (o.switch_tol < 0) o.switch_tol = 0;
    struct PrecisionGuard {
      fnocc_ctx *c;
      ~PrecisionGuard() { c->precision = FNOCC_FP64; }
    } guard{c};
    if (o.tol_res <= 0) o.tol_res = 1e-8;
    if (o.tol_e <= 0) o.tol_e = 1e-10;
    if (o.maxiter <= 0) o.maxiter = 200;
    Launch L = c->L();
    c->precision = FNOCC_FP64;
    prepare_hbar(c);  // T1 dressing and amplitude unpacking stay FP64
    c->precision = o.precision;
    int sigma_calls_mixed = 0;
    double split_best = INFINITY;  // split phase: best largest residual, and when it last halved
    int split_best_it = 0;
    size_t sz[3];
    eom_sizes(c, variant, sz);
    const long long dim = (long long)(sz[0] + sz[1] + sz[2]);
    // diagonal estimate and sector mask
    DevBuf dg, mk;
    dg.reserve(sizeof(double) * dim);
    mk.reserve(dim);
    size_t off = 0;
    for (int k = 0; k < 3; ++k) {
      int nh = kEom[variant][k][0], np = kEom[variant][k][1];
      eom_diag(L, c->fdiag.d(), c->o, nh, np, c->otab[nh].dev.as<int>(), c->otab[nh].count, c->vtab[np].dev.as<int>(),
               c->vtab[np].count, dg.d() + off);
      ms_mask(L, nh, np, c->otab[nh].dev.as<int>(), c->otab[nh].count, c->vtab[np].dev.as<int>(), c->vtab[np].count,
              kSectorMs2[variant], mk.as<unsigned char>() + off);
      off += sz[k];
    }
    std::vector<float> score;  // learned guess: predicted importance per element
    if (guess == FNOCC_GUESS_LEARNED) {
      const Mlp &net = *c->guess_model->net;
      if (net.device() != c->device) throw StatusError(FNOCC_E_INVALID, "guess network lives on another device");
      DevBuf feats, yout;
      feats.reserve(sizeof(float) * dim * kMlpFeatures);
      yout.reserve(sizeof(float) * dim * kMlpOutputs);
      eom_features_dev(c, variant, feats.as<float>());
      net.infer_bf16(feats.as<float>(), dim, yout.as<float>(), c->stream, c->mlp_scratch);
      // preconditioner: D + predicted correction (bounded)
      add_diag_correction(c->stream, dim, yout.as<float>(), kMlpOutputs, 1, 5.0, dg.d());
      std::vector<float> yh((size_t)dim * kMlpOutputs);
      FNOCC_CUDA(cudaMemcpyAsync(yh.data(), yout.p, sizeof(float) * yh.size(), cudaMemcpyDeviceToHost, c->stream));
      sync(c);
      score.resize(dim);
      for (long long i = 0; i < dim; ++i) score[i] = yh[(size_t)i * kMlpOutputs];
    }
    auto dgh = to_host(c, dg.d(), dim);
    std::vector<unsigned char> mkh(dim);
    copy_after(mkh.data(), mk.p, dim, cudaMemcpyDeviceToHost, c->stream);
    std::vector<long long> allowed, pref;
    for (long long i = 0; i < dim; ++i)
      if (mkh[i]) {
        allowed.push_back(i);
        if (guess == FNOCC_GUESS_DIAGONAL || i < (long long)sz[0]) pref.push_back(i);
      }
    if (allowed.empty()) throw StatusError(FNOCC_E_INVALID, "empty spin sector");
    int nr = std::min<long long>(nroots, (long long)allowed.size());
    int ng = o.nguess > 0 ? o.nguess : 2 * nr;
    ng = std::min<long long>(ng, (long long)allowed.size());
    int max_sub = o.max_sub > 0 ? o.max_sub : std::max(6 * nr, ng + 3 * nr);
    if (max_sub < std::max(ng, 2 * nr) + nr) max_sub = std::max(ng, 2 * nr) + nr;
    auto by_diag = [&](long long a, long long b) { return dgh[a] < dgh[b] || (dgh[a] == dgh[b] && a < b); };
    std::stable_sort(pref.begin(), pref.end(), by_diag);
    std::vector<long long> rest;
    {
      std::vector<unsigned char> inpref(dim, 0);
      for (auto i : pref) inpref[i] = 1;
      for (auto i : allowed)
        if (!inpref[i]) rest.push_back(i);
      std::stable_sort(rest.begin(), rest.end(), by_diag);
    }
    // unit guesses: KOOPMANS and LEARNED on the principal block only (its
    // determinants reach only the spin multiplicities whose states are
    // counted as roots), DIAGONAL on the whole space
    std::vector<long long> order(pref);
    if (guess == FNOCC_GUESS_LEARNED)  // highest predicted importance first
      std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) {
        return score[a] > score[b] || (score[a] == score[b] && a < b);
      });
    if ((long long)order.size() > ng) order.resize(ng);
    // Subspace vectors hold the sector's elements only (the allowed packed
    // indices in order: about a third of the packed space for the
    // M_s-conserving variants), so that the subspace of the largest spaces
    // fits next to the product's dense work tensors; products expand a
    // vector into the packed layout and take the sector's part back.
    const long long na = (long long)allowed.size();
    long long na0 = 0;  // allowed elements of the principal block (they come first)
    while (na0 < na && allowed[na0] < (long long)sz[0]) ++na0;
    DevBuf aidx, dgc;
    aidx.reserve(sizeof(long long) * na);
    FNOCC_CUDA(cudaMemcpyAsync(aidx.p, allowed.data(), sizeof(long long) * na, cudaMemcpyHostToDevice, c->stream));
    dgc.reserve(sizeof(double) * na);
    gather_idx(L, na, aidx.as<long long>(), dg.d(), dgc.d());
    sync(c);
    dg.release();
    mk.release();
    auto cpos = [&](long long full) {  // position of an allowed packed index in the sector
      return (long long)(std::lower_bound(allowed.begin(), allowed.end(), full) - allowed.begin());
    };
    DevBuf xfull, sfull;  // one product's input and output in the packed layout
    xfull.reserve(sizeof(double) * dim);
    sfull.reserve(sizeof(double) * dim);
    // elements outside the sector stay zero: the products only write the
    // allowed ones into xfull
    FNOCC_CUDA(cudaMemsetAsync(xfull.p, 0, sizeof(double) * dim, c->stream));
    const int cap = max_sub + nr + 1;
    DevBuf Vb, Sb, xr, rr, tmp;
    Vb.reserve(sizeof(double) * na * cap);
    Sb.reserve(sizeof(double) * na * cap);
    xr.reserve(sizeof(double) * na * nr);
    rr.reserve(sizeof(double) * na * nr);
    tmp.reserve(sizeof(double) * na);
    int kb = 0, sigma_calls = 0;
    std::vector<double> G;  // kb x kb, row-major, G[i][j] = V_i . S_j
    std::vector<double> G1;  // kb x kb, principal-block overlaps V_i[0:sz0] . V_j[0:sz0]
    auto vrow = [&](int i) { return Vb.d() + (size_t)i * na; };
    auto srow = [&](int i) { return Sb.d() + (size_t)i * na; };
    // Appends src, orthonormalised against the basis (Gram-Schmidt twice), and
    // its product: computed, or (restart) carried along linearly from sig_src.
    auto add_vector = [&](const double *src, const double *sig_src = nullptr) -> bool {
      double *dst = vrow(kb);
      double *sdst = srow(kb);
      FNOCC_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * na, cudaMemcpyDeviceToDevice, c->stream));
      if (sig_src)
        FNOCC_CUDA(cudaMemcpyAsync(sdst, sig_src, sizeof(double) * na, cudaMemcpyDeviceToDevice, c->stream));
      for (int pass = 0; pass < 2 && kb > 0; ++pass) {
        c->small.reserve(sizeof(double) * std::max(64, kb));
        multi_dot(L, na, dst, Vb.d(), na, kb, c->small.d(), c->red);
        auto d = to_host(c, c->small.d(), kb);
        for (auto &x : d) x = -x;
        combine_rows(c, na, Vb.d(), kb, d, dst, true);
        if (sig_src) combine_rows(c, na, Sb.d(), kb, d, sdst, true);
      }
      double amax, nrm;
      absmax_dev(c, na, dst, &amax, &nrm);
      if (!(nrm > 1e-10)) return false;
      axpby(L, na, 0.0, dst, 1.0 / nrm, dst);
      if (sig_src) {
        axpby(L, na, 0.0, sdst, 1.0 / nrm, sdst);
      } else {
        scatter_idx(L, na, aidx.as<long long>(), dst, xfull.d());
        sigma_dev(c, variant, xfull.d(), sfull.d(), c->eom_left);
        gather_idx(L, na, aidx.as<long long>(), sfull.d(), sdst);
        ++sigma_calls;
        if (c->precision != FNOCC_FP64) ++sigma_calls_mixed;
      }
      // extend G
      int k1 = kb + 1;
      std::vector<double> Gn((size_t)k1 * k1, 0.0);
      for (int i = 0; i < kb; ++i)
        for (int j = 0; j < kb; ++j) Gn[i * k1 + j] = G[i * kb + j];
      c->small.reserve(sizeof(double) * std::max(64, k1));
      multi_dot(L, na, srow(kb), Vb.d(), na, k1, c->small.d(), c->red);  // V_i . S_new
      auto col = to_host(c, c->small.d(), k1);
      for (int i = 0; i < k1; ++i) Gn[i * k1 + kb] = col[i];
      if (kb > 0) {
        multi_dot(L, na, vrow(kb), Sb.d(), na, kb, c->small.d(), c->red);  // V_new . S_j
        auto row = to_host(c, c->small.d(), kb);
        for (int j = 0; j < kb; ++j) Gn[kb * k1 + j] = row[j];
      }
      G.swap(Gn);
      std::vector<double> G1n((size_t)k1 * k1, 0.0);
      for (int i = 0; i < kb; ++i)
        for (int j = 0; j < kb; ++j) G1n[i * k1 + j] = G1[i * kb + j];
      multi_dot(L, na0, vrow(kb), Vb.d(), na, k1, c->small.d(), c->red);  // principal overlaps
      auto pc = to_host(c, c->small.d(), k1);
      for (int i = 0; i < k1; ++i) G1n[i * k1 + kb] = G1n[kb * k1 + i] = pc[i];
      G1.swap(G1n);
      kb = k1;
      return true;
    };
    auto add_unit = [&](long long full) {
      FNOCC_CUDA(cudaMemsetAsync(tmp.p, 0, sizeof(double) * na, c->stream));
      double one = 1.0;
      FNOCC_CUDA(cudaMemcpyAsync(tmp.d() + cpos(full), &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
      sync(c);
      return add_vector(tmp.d());
    };
    for (long long idx : order) add_unit(idx);
    // fewer unit guesses than ng: Krylov vectors (products of the basis stay
    // in the multiplicities reached so far), then the lowest-diagonal
    // remaining elements
    for (int src = 0; kb < ng && src < kb; ++src) add_vector(srow(src));
    for (size_t q = 0; kb < ng && q < rest.size(); ++q) add_unit(rest[q]);
    std::vector<double> theta(nr, 0.0), theta_old(nr, 0.0), norms(nr, 0.0);
    bool have_old = false, conv = false;
    int it, ncomplex = 0;
    for (it = 1; it <= o.maxiter; ++it) {
      std::vector<std::complex<double>> w, Y;
      eig_nonsym(kb, G, w, Y);
      std::vector<int> idx(kb);
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a].real() < w[b].real(); });
      {
        // roots are counted among Ritz vectors with principal-block weight:
        // states of other spin multiplicities (pure satellites, e.g. the
        // quintet 3h1p states of DIP) have none and appear only by rounding
        // (fewer principal states than roots: the lowest others fill up)
        std::vector<int> good, rest;
        for (int j : idx) {
          double yy = 0, wt = 0;
          for (int a = 0; a < kb; ++a) {
            const double ya = Y[(size_t)a * kb + j].real();
            yy += ya * ya;
            for (int b = 0; b < kb; ++b) wt += ya * G1[(size_t)a * kb + b] * Y[(size_t)b * kb + j].real();
          }
          (yy > 0 && wt / yy >= kMinPrincipalWeight ? good : rest).push_back(j);
        }
        std::vector<int> chosen(good.begin(), good.begin() + std::min<size_t>(good.size(), nr));
        for (size_t q = 0; (int)chosen.size() < nr && q < rest.size(); ++q) chosen.push_back(rest[q]);
        std::stable_sort(chosen.begin(), chosen.end(), [&](int a, int b) { return w[a].real() < w[b].real(); });
        for (size_t q = nr; q < good.size(); ++q) chosen.push_back(good[q]);
        idx = chosen;
      }
      ncomplex = 0;
      std::vector<std::vector<double>> ys(nr);
      for (int r = 0; r < nr; ++r) {
        int j = idx[r];
        theta[r] = w[j].real();
        if (std::fabs(w[j].imag()) > 1e-8) ++ncomplex;
        std::vector<double> y(kb);
        for (int i = 0; i < kb; ++i) y[i] = Y[(size_t)i * kb + j].real();
        // normalise the Ritz vector: basis is orthonormal, so |x| = |y|
        double nn = 0;
        for (double a : y) nn += a * a;
        nn = std::sqrt(nn);
        if (nn == 0) nn = 1;
        for (double &a : y) a /= nn;
        ys[r] = y;
        double *x = xr.d() + (size_t)r * na;
        double *res = rr.d() + (size_t)r * na;
        combine_rows(c, na, Vb.d(), kb, y, x, false);
        combine_rows(c, na, Sb.d(), kb, y, res, false);
        axpby(L, na, -theta[r], x, 1.0, res);
        double amax, nrm;
        absmax_dev(c, na, res, &amax, &nrm);
        if (!std::isfinite(nrm)) throw StatusError(FNOCC_E_NUMERIC, "NaN in Davidson residual");
        norms[r] = nrm;
      }
      if (c->precision != FNOCC_FP64 && o.switch_tol > 0) {
        double mx = 0;
        for (double x : norms) mx = std::max(mx, x);
        // refinement once every residual is below switch_tol, once the
        // largest residual has not halved for 25 iterations, or after half
        // of the iteration budget in split arithmetic (the roots selected by
        // principal weight can keep changing when satellites sit near the
        // weight threshold, and the split products' rounding is of the size
        // that moves them across it: FP64 then settles them)
        if (mx < 0.5 * split_best) {
          split_best = mx;
          split_best_it = it;
        }
        const bool stalled = it - split_best_it >= 25;
        if (mx < o.switch_tol || stalled || it >= std::max(8, o.maxiter / 2)) {
          // refinement: FP64 from here on, from a thick restart of the split
          // phase's subspace: the Ritz vectors of the chosen roots and of the
          // next candidates (2 nroots in all, as at every restart), their
          // products recomputed in FP64 (cached H-bar pieces too). With the
          // chosen roots' vectors alone the FP64 phase took about as many
          // iterations as a solve from the start.
          const int nkeep = std::min((int)idx.size(), 2 * nr);
          c->precision = FNOCC_FP64;
          ++c->hbar_version;
          DevBuf keep;
          keep.reserve(sizeof(double) * na * nkeep);
          for (int q = 0; q < nkeep; ++q) {
            std::vector<double> y(kb);
            double nn = 0;
            for (int i = 0; i < kb; ++i) {
              y[i] = Y[(size_t)i * kb + idx[q]].real();
              nn += y[i] * y[i];
            }
            nn = nn > 0 ? std::sqrt(nn) : 1.0;
            for (double &t : y) t /= nn;
            combine_rows(c, na, Vb.d(), kb, y, keep.d() + (size_t)q * na, false);
          }
          kb = 0;
          G.clear();
          G1.clear();
          for (int q = 0; q < nkeep; ++q) add_vector(keep.d() + (size_t)q * na);
          have_old = false;
          continue;
        }
      }
      const bool may_stop = c->precision == FNOCC_FP64 || o.switch_tol == 0;
      std::vector<bool> done(nr);
      bool all = true;
      for (int r = 0; r < nr; ++r) {
        // |d omega| against the nearest Ritz value of the previous iteration:
        // near-degenerate roots that swap rank do not restart the test
        double dth = INFINITY;
        for (int q = 0; q < nr; ++q) dth = std::min(dth, std::fabs(theta[r] - theta_old[q]));
        done[r] = may_stop && norms[r] < o.tol_res && have_old && dth < o.tol_e;
        all = all && done[r];
      }
      if (all) {
        conv = true;
        break;
      }
      theta_old = theta;
      have_old = true;
      int nnew = 0;
      for (int r = 0; r < nr; ++r)
        if (!done[r]) ++nnew;
      if (kb + nnew > max_sub) {
        // thick restart: keep the lowest nkeep Ritz vectors with their
        // products, formed as the same linear combinations (no new products)
        const int nkeep = std::min((int)idx.size(), 2 * nr);
        DevBuf kx, ks;
        kx.reserve(sizeof(double) * na * nkeep);
        ks.reserve(sizeof(double) * na * nkeep);
        for (int q = 0; q < nkeep; ++q) {
          int j = idx[q];
          std::vector<double> y(kb);
          for (int i = 0; i < kb; ++i) y[i] = Y[(size_t)i * kb + j].real();
          double nn = 0;
          for (double t : y) nn += t * t;
          nn = std::sqrt(nn);
          if (nn == 0) nn = 1;
          for (double &t : y) t /= nn;
          combine_rows(c, na, Vb.d(), kb, y, kx.d() + (size_t)q * na, false);
          combine_rows(c, na, Sb.d(), kb, y, ks.d() + (size_t)q * na, false);
        }
        kb = 0;
        G.clear();
        G1.clear();
        for (int q = 0; q < nkeep; ++q) add_vector(kx.d() + (size_t)q * na, ks.d() + (size_t)q * na);
      }
      for (int r = 0; r < nr; ++r) {
        if (done[r]) continue;
        precondition(L, na, rr.d() + (size_t)r * na, dgc.d(), theta[r], nullptr, tmp.d());
        add_vector(tmp.d());
      }
    }
    if (!conv) it = o.maxiter;
    // results
    for (int r = 0; r < nroots; ++r) {
      double th = r < nr ? theta[r] : NAN;
      energies[r] = c->e_ref + c->e_corr + th;
      if (omegas) omegas[r] = th;
    }
    // root vectors in the packed layout (zero outside the sector)
    Vb.release();
    Sb.release();
    c->eom_vecs.reserve(sizeof(double) * dim * nr);
    FNOCC_CUDA(cudaMemsetAsync(c->eom_vecs.p, 0, sizeof(double) * dim * nr, c->stream));
    for (int r = 0; r < nr; ++r)
      scatter_idx(L, na, aidx.as<long long>(), xr.d() + (size_t)r * na, c->eom_vecs.d() + (size_t)r * dim);
    sync(c);
    c->last_variant = variant;
    c->last_nroots = nr;
    c->last_dim = dim;
    double secs = timer.s();
    if (out) {
      out->iters = it;
      out->sigma_calls = sigma_calls;
      out->seconds = secs;
      out->seconds_per_iter = secs / std::max(1, it);
      out->complex_roots = ncomplex;
      double mx = 0;
      for (double x : norms) mx = std::max(mx, x);
      out->res_max = mx;
      out->sigma_calls_mixed = sigma_calls_mixed;
      out->guess_used = guess;
    }
    return conv ? FNOCC_OK : FNOCC_NOT_CONVERGED;
  });
}

fnocc_status eom_ccsdt_solve_left(fnocc_ctx *c, int variant, int nroots, int guess, const eom_options *opt,
                                  double *energies, double *omegas, eom_info *out) {
  if (!c) return FNOCC_E_INVALID;
  struct LeftGuard {
    fnocc_ctx *c;
    ~LeftGuard() { c->eom_left = false; }
  } guard{c};
  c->eom_left = true;
  return eom_ccsdt_solve(c, variant, nroots, guess, opt, energies, omegas, out);
}

fnocc_status eom_ccsdt_solve(fnocc_ctx *c, int variant, int nroots, int guess, const eom_options *opt,
                             double *energies, double *omegas, eom_info *out) {
  fnocc_status st = eom_solve_once(c, variant, nroots, guess, opt, energies, omegas, out);
  if (guess == FNOCC_GUESS_LEARNED && st == FNOCC_NOT_CONVERGED) {
    // plain Davidson from the Koopmans guess judges: roots never depend on the network
    eom_info first{};
    if (out) first = *out;
    st = eom_solve_once(c, variant, nroots, FNOCC_GUESS_KOOPMANS, opt, energies, omegas, out);
    if (out) {
      out->sigma_calls += first.sigma_calls;
      out->sigma_calls_mixed += first.sigma_calls_mixed;
      out->seconds += first.seconds;
      out->iters += first.iters;
    }
  }
  return st;
}

fnocc_status fnocc_eom_features(fnocc_ctx *c, int variant, float *features) {
  if (!c || !features) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (variant < 0 || variant >= kEomVariants) throw StatusError(FNOCC_E_INVALID, "bad variant");
    require_ham(c);
    FNOCC_CUDA(cudaSetDevice(c->device));
    size_t sz[3];
    eom_sizes(c, variant, sz);
    const size_t dim = sz[0] + sz[1] + sz[2];
    DevBuf f;
    f.reserve(sizeof(float) * dim * kMlpFeatures);
    eom_features_dev(c, variant, f.as<float>());
    FNOCC_CUDA(cudaMemcpyAsync(features, f.p, sizeof(float) * dim * kMlpFeatures, cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    return FNOCC_OK;
  });
}

namespace {

// exact diagonal elements H-bar_mumu at the packed indices idx (all of the
// space when idx is null), one product with a unit vector per element inside
// the sector; out[q] belongs to idx[q] (to element q without idx)
void eom_diagonal_elements(fnocc_ctx *c, int variant, long long n, const long long *idx, double *out) {
  if (variant < 0 || variant >= kEomVariants) throw StatusError(FNOCC_E_INVALID, "bad variant");
  require_ham(c);
  FNOCC_CUDA(cudaSetDevice(c->device));
  size_t sz[3];
  eom_sizes(c, variant, sz);
  const long long dim = (long long)(sz[0] + sz[1] + sz[2]);
  if (!idx) n = dim;
  for (long long q = 0; idx && q < n; ++q)
    if (idx[q] < 0 || idx[q] >= dim) throw StatusError(FNOCC_E_INVALID, "element index out of range");
  prepare_hbar(c);
  c->precision = FNOCC_FP64;
  Launch L = c->L();
  DevBuf mk, x, s, dd;
  mk.reserve(dim);
  size_t off = 0;
  for (int k = 0; k < 3; ++k) {
    const int nh = kEom[variant][k][0], np = kEom[variant][k][1];
    ms_mask(L, nh, np, c->otab[nh].dev.as<int>(), c->otab[nh].count, c->vtab[np].dev.as<int>(), c->vtab[np].count,
            kSectorMs2[variant], mk.as<unsigned char>() + off);
    off += sz[k];
  }
  std::vector<unsigned char> mkh(dim);
  copy_after(mkh.data(), mk.p, dim, cudaMemcpyDeviceToHost, c->stream);
  x.reserve(sizeof(double) * dim);
  s.reserve(sizeof(double) * dim);
  dd.reserve(sizeof(double) * std::max<long long>(n, 1));
  FNOCC_CUDA(cudaMemsetAsync(x.p, 0, sizeof(double) * dim, c->stream));
  FNOCC_CUDA(cudaMemsetAsync(dd.p, 0, sizeof(double) * std::max<long long>(n, 1), c->stream));
  const double one = 1.0, zero = 0.0;
  for (long long q = 0; q < n; ++q) {
    const long long i = idx ? idx[q] : q;
    if (!mkh[i]) continue;
    FNOCC_CUDA(cudaMemcpyAsync(x.d() + i, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    sigma_dev(c, variant, x.d(), s.d());
    FNOCC_CUDA(cudaMemcpyAsync(dd.d() + q, s.d() + i, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    FNOCC_CUDA(cudaMemcpyAsync(x.d() + i, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  if (n > 0) copy_after(out, dd.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
}

}  // namespace

fnocc_status fnocc_eom_diagonal(fnocc_ctx *c, int variant, double *diag) {
  if (!c || !diag) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    eom_diagonal_elements(c, variant, 0, nullptr, diag);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_eom_diagonal_at(fnocc_ctx *c, int variant, long long n, const long long *idx, double *out) {
  if (!c || n < 0 || (n > 0 && (!idx || !out))) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (n > 0) eom_diagonal_elements(c, variant, n, idx, out);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_set_guess_model(fnocc_ctx *c, fnocc_mlp *mlp) {
  if (!c) return FNOCC_E_INVALID;
  c->guess_model = mlp;
  return FNOCC_OK;
}

fnocc_status fnocc_multi_dot(fnocc_ctx *c, const double *x, const double *Y, size_t n, size_t ld, int nvec,
                             double *dots) {
  if (!c) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    if (!x || !Y || !dots || nvec <= 0 || n == 0 || ld < n) throw StatusError(FNOCC_E_INVALID, "bad multi_dot arguments");
    FNOCC_CUDA(cudaSetDevice(c->device));
    multi_dot(c->L(), (long long)n, x, Y, (long long)ld, nvec, dots, c->red);
    sync(c);
    return FNOCC_OK;
  });
}

fnocc_status fnocc_get_block(fnocc_ctx *c, int which, int root, double *buf, size_t len) {
  if (!c || !buf) return FNOCC_E_INVALID;
  return guarded(c, [&]() -> fnocc_status {
    require_ham(c);
    if (which >= 1 && which <= 3) {
      if (!c->have_amps) throw StatusError(FNOCC_E_STATE, "no amplitudes");
      size_t off = (which >= 2 ? c->nt[1] : 0) + (which >= 3 ? c->nt[2] : 0);
      if (len != c->nt[which]) throw StatusError(FNOCC_E_INVALID, "length mismatch");
      copy_after(buf, c->tpk.d() + off, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream);
      return FNOCC_OK;
    }
    if (which >= 11 && which <= 13) {
      if (c->last_variant < 0 || root < 0 || root >= c->last_nroots) throw StatusError(FNOCC_E_STATE, "no such EOM root");
      size_t sz[3];
      eom_sizes(c, c->last_variant, sz);
      int k = which - 11;
      size_t off = (k >= 1 ? sz[0] : 0) + (k >= 2 ? sz[1] : 0);
      if (len != sz[k]) throw StatusError(FNOCC_E_INVALID, "length mismatch");
      copy_after(buf, c->eom_vecs.d() + (size_t)root * c->last_dim + off, sizeof(double) * len,
                 cudaMemcpyDeviceToHost, c->stream);
      return FNOCC_OK;
    }
    throw StatusError(FNOCC_E_INVALID, "unknown block");
  });
}

fnocc_status fnocc_batch_solve(int device, int nsys, const fnocc_system *systems, int nvariants, const int *variants,
                               int nroots, const ccsdt_options *cc_opt, const eom_options *eom_opt, int nworkers,
                               double *omegas, fnocc_system_result *results) {
  if (nsys <= 0 || !systems || nvariants <= 0 || !variants || nroots <= 0 || !omegas) return FNOCC_E_INVALID;
  for (int k = 0; k < nvariants; ++k)
    if (variants[k] < 0 || variants[k] >= kEomVariants) return FNOCC_E_INVALID;
  for (int s = 0; s < nsys; ++s)
    if (!systems[s].h || !systems[s].eri || systems[s].n <= 1 || systems[s].nocc <= 0 || systems[s].nocc >= systems[s].n)
      return FNOCC_E_INVALID;
  if (nworkers <= 0) nworkers = 4;
  nworkers = std::min(nworkers, nsys);
  // largest systems first (cost grows steeply with the orbital count)
  std::vector<int> order(nsys);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return systems[a].n > systems[b].n; });
  std::atomic<int> next(0);
  std::vector<fnocc_status> st(nsys, FNOCC_OK);
  std::vector<char> attempted(nsys, 0);
  std::atomic<int> create_status(FNOCC_OK);
  // a worker whose context cannot be created leaves the queue to the others;
  // systems no worker reached get that worker's status after the join
  auto worker = [&]() {
    fnocc_ctx *c = nullptr;
    const fnocc_status cs = fnocc_create(&c, device, nullptr);
    if (cs != FNOCC_OK) {
      create_status.store(cs);
      return;
    }
    for (int q; (q = next.fetch_add(1)) < nsys;) {
      const int s = order[q];
      attempted[s] = 1;
      const fnocc_system &sys = systems[s];
      Timer timer;
      fno_options fo{FNOCC_CRIT_ABS, sys.nkeep, 200, 1e-12, 1e-10};
      fno_info fi{};
      ccsdt_info ci{};
      std::string msg;
      fnocc_status worst = fno_truncate(c, sys.h, sys.eri, sys.n, sys.nocc, sys.occ_threshold, &fo, &fi, nullptr);
      if (worst != FNOCC_OK) msg = c->err;
      int sig = 0;
      if (worst >= 0) {
        fnocc_status cs = ccsdt_solve(c, cc_opt, &ci);
        if (cs != FNOCC_OK) {
          worst = cs;
          if (msg.empty()) msg = cs == FNOCC_NOT_CONVERGED ? "CCSDT did not converge" : c->err;
        }
        if (cs >= 0)
          for (int k = 0; k < nvariants; ++k) {
            eom_info ei{};
            std::vector<double> en(nroots);
            fnocc_status es = eom_ccsdt_solve(c, variants[k], nroots, FNOCC_GUESS_KOOPMANS, eom_opt, en.data(),
                                              omegas + ((size_t)s * nvariants + k) * nroots, &ei);
            sig += ei.sigma_calls;
            if (es != FNOCC_OK && msg.empty())
              msg = es == FNOCC_NOT_CONVERGED ? "EOM variant " + std::to_string(variants[k]) + " did not converge"
                                              : c->err;
            if (es < 0 || (es != FNOCC_OK && worst >= 0)) worst = es;
          }
      }
      st[s] = worst;
      if (results) {
        results[s].status = worst;
        results[s].nkept = fi.nkept;
        results[s].e_rhf = fi.e_rhf;
        results[s].e_ccsdt = ci.e_tot;
        results[s].ccsdt_iters = ci.iters;
        results[s].sigma_calls = sig;
        results[s].seconds = timer.s();
        std::snprintf(results[s].message, sizeof(results[s].message), "%s", msg.c_str());
      }
    }
    fnocc_destroy(c);
  };
  std::vector<std::thread> pool;
  try {
    for (int w = 0; w < nworkers; ++w) pool.emplace_back(worker);
  } catch (const std::exception &) {
    // no more threads: the started workers drain the queue; none started, this one does
  }
  if (pool.empty()) worker();
  for (auto &t : pool) t.join();
  for (int s = 0; s < nsys; ++s)
    if (!attempted[s]) {
      st[s] = create_status.load() != FNOCC_OK ? (fnocc_status)create_status.load() : FNOCC_E_CUDA;
      if (results) {
        results[s] = fnocc_system_result{st[s], 0, 0.0, 0.0, 0, 0, 0.0, {0}};
        std::snprintf(results[s].message, sizeof(results[s].message), "no worker context could be created");
      }
    }
  fnocc_status out = FNOCC_OK;
  for (int s = 0; s < nsys; ++s)
    if (st[s] < 0) return st[s];
    else if (st[s] != FNOCC_OK) out = st[s];
  return out;
}

namespace {

// kind 0: CCSDT rank out_comp; 1: right EOM block; 2: left EOM block
bool equation_of(int kind, int variant, int out_comp, int in_comp, Equation *eq) {
  if (kind == 0) {
    if (out_comp < 0 || out_comp > 3) return false;
    *eq = cc_equation(out_comp);
    return true;
  }
  if ((kind != 1 && kind != 2) || variant < 0 || variant >= kEomVariants || out_comp < 0 || out_comp > 2 ||
      in_comp < 0 || in_comp > 2)
    return false;
  *eq = kind == 1 ? eom_equation(variant, out_comp, in_comp) : eom_left_equation(variant, out_comp, in_comp);
  return true;
}

}  // namespace

long fnocc_equation_text(int kind, int variant, int out_comp, int in_comp, char *buf, size_t len) {
  try {
    Equation eq;
    if (!equation_of(kind, variant, out_comp, in_comp, &eq)) return -1;
    std::string s = equation_to_string(eq);
    if (buf && len > 0) {
      size_t n = std::min(len - 1, s.size());
      std::memcpy(buf, s.data(), n);
      buf[n] = 0;
    }
    return (long)s.size();
  } catch (...) {
    return -1;
  }
}

long fnocc_plan_selfcheck(int kind, int variant, int out_comp, int in_comp, int o, int v, double max_work) {
  try {
    if (o <= 0 || v <= 0 || o > 64 || v > 128) return -1;
    int rd[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    if (kind == 0 && out_comp >= 0 && out_comp <= 3) {
      ExecEquation e(cc_equation(out_comp), o, v, rd, 0.0, 0.0, 0, true);
      return (long)e.self_check(max_work);
    }
    Equation eq;
    if (kind == 0 || !equation_of(kind, variant, out_comp, in_comp, &eq)) return -1;
    for (int k = 0; k < 3; ++k) {
      rd[k][0] = kEom[variant][k][0];
      rd[k][1] = kEom[variant][k][1];
    }
    ExecEquation e(eq, o, v, rd, kSigmaAmortize, kCacheCapDoubles, kSectorMs2[variant], true);
    return (long)e.self_check(max_work);
  } catch (...) {
    return -1;
  }
}

fnocc_status fnocc_plan_stats(int kind, int variant, int out_comp, int in_comp, int o, int v, double *stats) {
  try {
    if (!stats || o <= 0 || v <= 0 || o > 64 || v > 128) return FNOCC_E_INVALID;
    Equation eq;
    if (!equation_of(kind, variant, out_comp, in_comp, &eq)) return FNOCC_E_INVALID;
    int rd[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    if (kind != 0)
      for (int k = 0; k < 3; ++k) {
        rd[k][0] = kEom[variant][k][0];
        rd[k][1] = kEom[variant][k][1];
      }
    ExecEquation e(eq, o, v, rd, kind == 0 ? 0.0 : kSigmaAmortize, kind == 0 ? 0.0 : kCacheCapDoubles,
                   kind == 0 ? 0 : kSectorMs2[variant], true);
    e.stats(stats);
    return FNOCC_OK;
  } catch (...) {
    return FNOCC_E_INVALID;
  }
}

long fnocc_plan_text(int kind, int variant, int out_comp, int in_comp, int o, int v, double amortize, char *buf,
                     size_t len) {
  try {
    if (o <= 0 || v <= 0) return -1;
    Equation eq;
    if (!equation_of(kind, variant, out_comp, in_comp, &eq)) return -1;
    std::ostringstream os;
    os.precision(17);
    auto groups = [&](const std::vector<DimGroup> &gs) {
      os << " " << gs.size();
      for (auto &g : gs) {
        os << " " << g.space << ":" << g.k << ":" << (g.packed ? 1 : 0) << ":";
        for (size_t i = 0; i < g.labels.size(); ++i) os << (i ? "," : "") << g.labels[i];
      }
    };
    std::vector<TermPlan> raw;
    for (auto &t : eq.terms) raw.push_back(plan_term(t, eq.nh, eq.np, o, v, amortize, double(1LL << 28)));
    std::vector<TermPlan> plans = fuse_plans(raw, amortize);
    os << eq.nh << " " << eq.np << " " << plans.size() << "\n";
    for (auto &p : plans) {
      os << "TERM " << p.steps.size() << " " << p.inter_dims.size() << "\n";
      for (size_t i = 0; i < p.inter_dims.size(); ++i) {
        os << "INTER " << i;
        groups(p.inter_dims[i]);
        os << "\n";
      }
      for (auto &s : p.steps) {
        os << "STEP " << s.a.kind << " " << s.a.inter << " " << s.b.kind << " " << s.b.inter << " " << (s.to_output ? 1 : 0)
           << " " << s.out_inter << " " << (s.constant ? 1 : 0) << " " << s.alpha;
        os << " A";
        for (int l : s.a.labels) os << " " << l;
        os << " B";
        for (int l : s.b.labels) os << " " << l;
        os << " M";
        groups(s.mg);
        os << " K";
        groups(s.kg);
        os << " N";
        groups(s.ng);
        os << "\n";
      }
    }
    std::string str = os.str();
    if (buf && len > 0) {
      size_t n = std::min(len - 1, str.size());
      std::memcpy(buf, str.data(), n);
      buf[n] = 0;
    }
    return (long)str.size();
  } catch (...) {
    return -1;
  }
}

double xfno_extrapolate(const double *f, const double *e, int npts) {
  if (!f || !e || npts < 1) return NAN;
  double mf = 0, me = 0;
  for (int i = 0; i < npts; ++i) {
    mf += f[i];
    me += e[i];
  }
  mf /= npts;
  me /= npts;
  double sff = 0, sfe = 0;
  for (int i = 0; i < npts; ++i) {
    sff += (f[i] - mf) * (f[i] - mf);
    sfe += (f[i] - mf) * (e[i] - me);
  }
  if (sff == 0) return me;
  double slope = sfe / sff;
  return me + slope * (1.0 - mf);
}

}  // extern "C"
