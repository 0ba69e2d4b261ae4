// Execution of planned equations on the device: offset tables, intermediate
// scratch and the launch sequence of one projected equation.
#pragma once
#include "common.hpp"
#include "planner.hpp"

#include <initializer_list>
#include <memory>

namespace fnocc {

// Device pointers of the operands an equation reads.
struct Operands {
  const double *f = nullptr;    // n x n one-body operator (n = o + v), full
  const double *v = nullptr;    // n^4 antisymmetrised two-body operator, full
  const double *t2 = nullptr;   // dense [o,o,v,v]
  const double *t3 = nullptr;   // dense [o,o,o,v,v,v]
  const double *r[3] = {nullptr, nullptr, nullptr};  // dense EOM components
  // element counts of the buffers above (checked against every index map)
  long long f_size = 0, v_size = 0, t2_size = 0, t3_size = 0, r_size[3] = {0, 0, 0};
};

// One spin-allowed block of a step: for every M, K and N group a contiguous
// segment (start, length) of its spin-sorted tuple list.
struct SubGemm {
  std::vector<std::pair<long long, long long>> mseg, kseg, nseg;
  long long M = 0, N = 0, K = 0;
};

struct ExecStep {
  int a_kind, a_inter, b_kind, b_inter;
  bool blocked = false;          // run as spin-allowed sub-GEMMs
  std::vector<SubGemm> blocks;
  bool constant;   // R-independent: run once per H-bar version into the cache
  bool zero_first; // first writer of its intermediate: zero it before the step
  bool to_output;
  int out_inter;
  long long M, N, K;
  double alpha;
  DMap arow, acol, brow, bcol, crow, ccol;
  // grouped launch (every binary step whose output has more than 256
  // elements): one task per spin-allowed (row block, column block) pair with
  // its reduction blocks concatenated, flat offset tables, and one launch
  // descriptor per tile shape
  bool grouped = false;
  struct TaskRef {
    long long M, N, K, arow, acol, brow, bcol, crow, ccol;  // offsets into the flat table buffer
  };
  std::vector<TaskRef> tasks;
  GroupedLaunch gl[kGShapesAll];
  long long gmax_a = 0, gmax_b = 0, gmax_c = 0;  // largest row + column offset per operand
  int default_shape = 0;                          // least padded work per busy SM
  int bf16_shape = kGShapeBf16;                   // mma.sync split tile with the least staged work per busy SM
  int tc_shape = kGShapeTc;                       // tcgen05 BF16x3 tile with the least staged work per busy SM
  int tc_shape_alt = kGShapeTc;                   // the best one of the other orientation (lanes on B's columns)
  int tcp_shape = -1;                             // tcgen05 panel tile with the least padded work (-1: panels too large)
  int bf16x3_shape = kGShapeBf16;                 // BF16x3 default: the better of the two estimates
  // BF16x3 steps above 1e8 padded flops: the mma.sync and the tcgen05 tile
  // are timed once each, then the faster is kept
  struct Trial {
    float ms[kGShapesAll] = {0};  // 0 untimed, < 0 in flight
    int pending = -1;             // event pair of this step, -1 none yet
  } mixed_tune;
  int tuned_mixed = -1;
  std::vector<int> cand;                          // FP64 shapes worth timing, best estimate first
  // tile-shape autotuning of large FP64 steps: every candidate is timed once,
  // then the fastest is kept
  int tuned_shape = -1;
  float trial_ms[kGShapes] = {0};  // 0 untimed, < 0 in flight
  int pending = -1;                // index of this step's event pair, -1 none yet
};

struct ExecTerm {
  std::vector<ExecStep> steps;
  std::vector<long long> inter_off;   // offsets (doubles) in scratch, or in the cache if cached
  std::vector<long long> inter_size;
  std::vector<char> inter_cached;
};

// One equation <mu_out| ... |0> compiled for fixed (o, v) and operand shapes.
class ExecEquation {
 public:
  // rdims: (nh, np) of the three EOM input components (ignored for CC)
  // amortize > 0: R-independent steps are cached (see plan_term)
  // r_charge: 2*M_s change of the EOM vectors (their spin sector); 0 for CC.
  // host_only: tables and launch descriptors stay in host memory (no
  // device needed; the plan cannot run, only self_check it)
  // sms: streaming multiprocessors of the device the plan runs on (reduction
  // splits and the wave model of the shape choice)
  ExecEquation(const Equation &eq, int o, int v, const int rdims[3][2], double amortize = 0.0,
               double cache_cap = 0.0, int r_charge = 0, bool host_only = false, int sms = 152);
  // host-only plans: number of inconsistencies between the grouped tasks of
  // every tile shape and the spin-allowed blocks (steps above max_work
  // multiply-adds skipped); 0 = consistent
  long long self_check(double max_work) const;
  // plan statistics of the FP64 grouped steps at their estimated tile
  // shapes (no device needed): see fnocc_plan_stats
  void stats(double out[10]) const;
  // Y (dense output accumulator [o^nh v^np]) += sum of terms. version: the
  // cached R-independent intermediates are recomputed when it changes.
  void run(const Launch &L, const Operands &ops, double *Y, long long y_size, DevBuf &scratch,
           uint64_t version = 0);
  // true when a run with this version would recompute the cached
  // R-independent intermediates
  bool needs_refresh(uint64_t version) const { return cache_need_ > 0 && version != cache_version_; }
  // true while a run under L would still time candidate tile shapes
  bool tuning_pending(const Launch &L) const;
  const void *cache_ptr() const { return cache_.p; }
  long long scratch_doubles() const { return scratch_need_; }
  long long cache_doubles() const { return cache_need_; }
  double flops() const { return flops_; }              // per run, cached steps excluded
  double cached_flops() const { return cached_flops_; }  // once per version
  ~ExecEquation();
  // autotuning switch for all equations (on by default)
  static bool autotune;
  int nh() const { return nh_; }
  int np() const { return np_; }
  size_t nterms() const { return terms_.size(); }

 private:
  void build_launches(const std::vector<long long> &flat_host);
  // one timing round of a step's candidate shapes: reads the trial of the
  // previous run, then launches the next untimed candidate between an event
  // pair of the step's own (read on a later run), or, once all are timed,
  // keeps the fastest in `tuned` and launches it
  void tune_launch(const Launch &L, ExecStep::Trial &tr, const std::vector<int> &cand, int &tuned,
                   const ExecStep &s, const double *A, const double *B, double *C);
  int nh_, np_, o_, v_;
  int sms_ = 152;
  bool host_only_ = false;
  std::vector<long long> host_tables_, host_flat_;
  std::vector<GTask> host_gt_;
  std::vector<int> host_sid_;
  std::vector<ExecTerm> terms_;
  DevBuf tables_;
  DevBuf flat_;    // flat offset tables of the grouped steps
  DevBuf gtasks_;  // GTask arrays and split-task lists of every step and shape
  DevBuf cache_;
  std::vector<cudaEvent_t> tune_events_;  // two per tuned step
  int tune_count_ = 0;
  uint64_t cache_version_ = ~0ULL;
  long long scratch_need_ = 0, cache_need_ = 0;
  double flops_ = 0, cached_flops_ = 0;
};

// Sorted index tuples (lexicographic) of k out of n, as a device int table.
struct TupleTable {
  int n = 0, k = 0;
  long long count = 0;
  DevBuf dev;
  // lexicographic rank of a sorted tuple c: sum_i S_i(c_i) - S_i(c_{i-1} + 1)
  // with S_i(x) = sum_{j < x} C(n-1-j, k-1-i) stored at rank[i * (n+1) + x]
  DevBuf rankdev;
  const long long *rank() const { return rankdev.as<long long>(); }
  void build(int n, int k);
};

long long binom_ll(int n, int k);

}  // namespace fnocc
