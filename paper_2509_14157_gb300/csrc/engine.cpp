// Compiles planned terms (planner.cpp) into offset tables and launches them
// through the gather-GEMM-scatter kernel (kernels.cu).
#include "engine.hpp"

#include <algorithm>
#include <map>

namespace fnocc {

long long binom_ll(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
  return r;
}

void TupleTable::build(int n_, int k_) {
  n = n_;
  k = k_;
  count = binom_ll(n, k);
  std::vector<int> host;
  host.reserve((size_t)std::max<long long>(count, 1) * std::max(k, 1));
  std::vector<int> cur(k);
  for (int i = 0; i < k; ++i) cur[i] = i;
  if (count > 0) {
    while (true) {
      for (int i = 0; i < k; ++i) host.push_back(cur[i]);
      int i = k - 1;
      while (i >= 0 && cur[i] == n - k + i) --i;
      if (i < 0) break;
      ++cur[i];
      for (int j = i + 1; j < k; ++j) cur[j] = cur[j - 1] + 1;
    }
  }
  if (host.empty()) host.push_back(0);
  dev.reserve(host.size() * sizeof(int));
  FNOCC_CUDA(cudaMemcpy(dev.p, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice));
}

namespace {

// Storage description of an operand: a list of dimensions, each holding one
// label (plain index) or a packed group of labels stored as sorted tuples.
struct SDim {
  std::vector<int> labels;
  bool packed = false;
  long long size = 0, stride = 0, base = 0;  // base: offset of the label's space (full tensors)
};

struct Storage {
  std::vector<SDim> dims;
  long long total() const {
    long long t = 1;
    for (auto &d : dims) t *= d.size;
    return t;
  }
};

void finish_strides(Storage &s) {
  long long st = 1;
  for (int i = (int)s.dims.size() - 1; i >= 0; --i) {
    s.dims[i].stride = st;
    st *= s.dims[i].size;
  }
}

Storage dense_storage(const std::vector<int> &labels, int o, int v) {
  Storage s;
  for (int lab : labels) {
    SDim d;
    d.labels = {lab};
    d.size = lab_space(lab) == SP_O ? o : v;
    s.dims.push_back(d);
  }
  finish_strides(s);
  return s;
}

Storage full_storage(const std::vector<int> &labels, int o, int v) {
  Storage s;
  for (int lab : labels) {
    SDim d;
    d.labels = {lab};
    d.size = o + v;
    d.base = lab_space(lab) == SP_O ? 0 : o;
    s.dims.push_back(d);
  }
  finish_strides(s);
  return s;
}

Storage group_storage(const std::vector<DimGroup> &groups, int o, int v) {
  Storage s;
  for (auto &g : groups) {
    int n = g.space == SP_O ? o : v;
    SDim d;
    d.labels = g.labels;
    d.packed = g.packed && g.k >= 2;
    d.size = d.packed ? binom_ll(n, g.k) : [&] { long long t = 1; for (int j = 0; j < g.k; ++j) t *= n; return t; }();
    if (!d.packed && g.k != 1) throw std::runtime_error("engine: unpacked multi-label dimension");
    s.dims.push_back(d);
  }
  finish_strides(s);
  return s;
}

// Output accumulator: externals in id order (holes then particles).
Storage output_storage(int nh, int np, int o, int v) {
  std::vector<int> labs;
  for (int k = 0; k < nh; ++k) labs.push_back(make_label(k, SP_O));
  for (int k = 0; k < np; ++k) labs.push_back(make_label(nh + k, SP_V));
  return dense_storage(labs, o, v);
}

struct TableBuilder {
  std::vector<long long> host;
  struct Pending { DMap *map; std::vector<long long> offs; };
  std::vector<Pending> pend;

  // appends the tables of `groups` over storage `s` and records a map to fix up
  long long add(DMap *map, const std::vector<DimGroup> &groups, const Storage &s, int o, int v) {
    if ((int)groups.size() > kMaxGroups) throw std::runtime_error("engine: too many dimension groups");
    map->ng = (int)groups.size();
    map->maxoff = 0;
    Pending p;
    p.map = map;
    long long total = 1;
    for (size_t g = 0; g < groups.size(); ++g) {
      const DimGroup &dg = groups[g];
      int n = dg.space == SP_O ? o : v;
      p.offs.push_back((long long)host.size());
      long long cnt = 0;
      // a packed storage dimension is read only as the same packed group
      const SDim *whole = nullptr;
      for (auto &d : s.dims)
        if (d.packed && d.labels == dg.labels) whole = &d;
      if (whole) {
        if (!dg.packed) throw std::runtime_error("engine: packed storage read unpacked");
        for (long long r = 0; r < whole->size; ++r) host.push_back(r * whole->stride);
        cnt = whole->size;
      } else {
        std::vector<long long> st(dg.k), bs(dg.k);
        for (int j = 0; j < dg.k; ++j) {
          const SDim *hit = nullptr;
          for (auto &d : s.dims)
            if (!d.packed && d.labels.size() == 1 && d.labels[0] == dg.labels[j]) hit = &d;
          if (!hit) throw std::runtime_error("engine: label not addressable in operand storage");
          st[j] = hit->stride;
          bs[j] = hit->base;
        }
        std::vector<int> cur(dg.k);
        if (dg.packed) {
          for (int j = 0; j < dg.k; ++j) cur[j] = j;
          if (binom_ll(n, dg.k) > 0)
            while (true) {
              long long off = 0;
              for (int j = 0; j < dg.k; ++j) off += st[j] * (bs[j] + cur[j]);
              host.push_back(off);
              ++cnt;
              int i = dg.k - 1;
              while (i >= 0 && cur[i] == n - dg.k + i) --i;
              if (i < 0) break;
              ++cur[i];
              for (int j = i + 1; j < dg.k; ++j) cur[j] = cur[j - 1] + 1;
            }
        } else {
          long long tot = 1;
          for (int j = 0; j < dg.k; ++j) tot *= n;
          for (long long x = 0; x < tot; ++x) {
            long long rem = x, off = 0;
            for (int j = dg.k - 1; j >= 0; --j) {
              off += st[j] * (bs[j] + rem % n);
              rem /= n;
            }
            host.push_back(off);
            ++cnt;
          }
        }
      }
      map->n[g] = cnt;
      long long mx = 0;
      for (long long q = p.offs.back(); q < (long long)host.size(); ++q) mx = std::max(mx, host[q]);
      map->maxoff += mx;
      total *= cnt;
    }
    pend.push_back(p);
    return total;
  }

  // tables of `groups` addressing storage dims first_dim, first_dim+1, ... in
  // order (the producer of an intermediate writes its dims positionally)
  long long add_positional(DMap *map, const std::vector<DimGroup> &groups, const Storage &s, int first_dim) {
    if ((int)groups.size() > kMaxGroups) throw std::runtime_error("engine: too many dimension groups");
    if (first_dim + (int)groups.size() > (int)s.dims.size()) throw std::runtime_error("engine: positional dims");
    map->ng = (int)groups.size();
    map->maxoff = 0;
    Pending p;
    p.map = map;
    long long total = 1;
    for (size_t g = 0; g < groups.size(); ++g) {
      const SDim &d = s.dims[first_dim + g];
      const DimGroup &dg = groups[g];
      if (d.packed != (dg.packed && dg.k >= 2) || (int)d.labels.size() != dg.k)
        throw std::runtime_error("engine: producer dims do not match the intermediate");
      p.offs.push_back((long long)host.size());
      for (long long r = 0; r < d.size; ++r) host.push_back(r * d.stride);
      map->n[g] = d.size;
      map->maxoff += (d.size - 1) * d.stride;
      total *= d.size;
    }
    pend.push_back(p);
    return total;
  }

  void upload(DevBuf &buf) {
    if (host.empty()) host.push_back(0);
    buf.reserve(host.size() * sizeof(long long));
    FNOCC_CUDA(cudaMemcpy(buf.p, host.data(), host.size() * sizeof(long long), cudaMemcpyHostToDevice));
    const long long *base = buf.as<long long>();
    for (auto &p : pend)
      for (size_t g = 0; g < p.offs.size(); ++g) p.map->tab[g] = base + p.offs[g];
  }
};

}  // namespace

ExecEquation::ExecEquation(const Equation &eq, int o, int v, const int rdims[3][2], double amortize,
                           double cache_cap)
    : nh_(eq.nh), np_(eq.np), o_(o), v_(v) {
  TableBuilder tb;
  Storage outs = output_storage(nh_, np_, o, v);
  std::vector<TermPlan> raw;
  for (const Term &t : eq.terms) raw.push_back(plan_term(t, nh_, np_, o, v, amortize, cache_cap));
  std::vector<TermPlan> plans = fuse_plans(raw, amortize);
  terms_.reserve(plans.size());
  for (const TermPlan &plan : plans) {
    ExecTerm et;
    std::vector<char> cached(plan.inter_labels.size(), 0);
    for (const Step &s : plan.steps)
      if (!s.to_output && s.constant) cached[s.out_inter] = 1;
    long long off = 0;
    std::vector<Storage> inter_store;
    for (auto &dims : plan.inter_dims) inter_store.push_back(group_storage(dims, o, v));
    for (size_t i = 0; i < plan.inter_labels.size(); ++i) {
      long long sz = inter_store[i].total();
      if (cached[i]) {
        et.inter_off.push_back(cache_need_);
        cache_need_ += sz;
      } else {
        et.inter_off.push_back(off);
        off += sz;
      }
      et.inter_size.push_back(sz);
    }
    et.inter_cached = cached;
    scratch_need_ = std::max(scratch_need_, off);
    auto storage_of = [&](const Operand &op) -> Storage {
      switch (op.kind) {
        case TK_F:
        case TK_V:
          return full_storage(op.labels, o, v);
        case TK_INTERMEDIATE:
          return inter_store.at(op.inter);
        default:
          return dense_storage(op.labels, o, v);
      }
    };
    et.steps.reserve(plan.steps.size());
    std::vector<char> written(plan.inter_dims.size(), 0);
    for (const Step &s : plan.steps) {
      ExecStep x;
      x.zero_first = !s.to_output && !written[s.out_inter];
      if (!s.to_output) written[s.out_inter] = 1;
      x.a_kind = s.a.kind;
      x.a_inter = s.a.inter;
      x.b_kind = s.b.kind;
      x.b_inter = s.b.inter;
      x.constant = s.constant;
      x.to_output = s.to_output;
      x.out_inter = s.out_inter;
      x.alpha = s.alpha;
      Storage sa = storage_of(s.a);
      Storage sc = s.to_output ? outs : inter_store.at(s.out_inter);
      et.steps.push_back(x);
      ExecStep &e = et.steps.back();
      e.M = tb.add(&e.arow, s.mg, sa, o, v);
      if (s.to_output)
        tb.add(&e.crow, s.mg, sc, o, v);
      else
        tb.add_positional(&e.crow, s.mg, sc, 0);
      if (s.b.kind >= 0) {
        Storage sb = storage_of(s.b);
        e.K = tb.add(&e.acol, s.kg, sa, o, v);
        tb.add(&e.brow, s.kg, sb, o, v);
        e.N = tb.add(&e.bcol, s.ng, sb, o, v);
        if (s.to_output)
          tb.add(&e.ccol, s.ng, sc, o, v);
        else
          tb.add_positional(&e.ccol, s.ng, sc, (int)s.mg.size());
        (s.constant ? cached_flops_ : flops_) += 2.0 * double(e.M) * double(e.N) * double(e.K);
      } else {
        e.N = 1;
        e.K = 1;
        (s.constant ? cached_flops_ : flops_) += double(e.M);
      }
    }
    terms_.push_back(std::move(et));
  }
  (void)rdims;
  tb.upload(tables_);
}

void ExecEquation::run(const Launch &L, const Operands &ops, double *Y, long long y_size, DevBuf &scratch,
                       uint64_t version) {
  if (scratch_need_ > 0) scratch.reserve(sizeof(double) * (size_t)scratch_need_);
  const bool refresh = cache_need_ > 0 && version != cache_version_;
  if (cache_need_ > 0) cache_.reserve(sizeof(double) * (size_t)cache_need_);
  for (const ExecTerm &t : terms_) {
    auto ptr = [&](int kind, int inter) -> const double * {
      switch (kind) {
        case TK_F: return ops.f;
        case TK_V: return ops.v;
        case TK_T2: return ops.t2;
        case TK_T3: return ops.t3;
        case TK_R1: return ops.r[0];
        case TK_R2: return ops.r[1];
        case TK_R3: return ops.r[2];
        case TK_INTERMEDIATE: return (t.inter_cached[inter] ? cache_.d() : scratch.d()) + t.inter_off[inter];
        default: throw std::runtime_error("engine: unknown operand kind");
      }
    };
    auto size = [&](int kind, int inter) -> long long {
      switch (kind) {
        case TK_F: return ops.f_size;
        case TK_V: return ops.v_size;
        case TK_T2: return ops.t2_size;
        case TK_T3: return ops.t3_size;
        case TK_R1: return ops.r_size[0];
        case TK_R2: return ops.r_size[1];
        case TK_R3: return ops.r_size[2];
        case TK_INTERMEDIATE: return t.inter_size[inter];
        default: return 0;
      }
    };
    for (const ExecStep &s : t.steps) {
      if (s.constant && !refresh) continue;  // cached and still valid
      double *C;
      long long csize;
      if (s.to_output) {
        C = Y;
        csize = y_size;
      } else {
        csize = t.inter_size[s.out_inter];
        C = (t.inter_cached[s.out_inter] ? cache_.d() : scratch.d()) + t.inter_off[s.out_inter];
        if (s.zero_first) FNOCC_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * t.inter_size[s.out_inter], L.stream));
      }
      const double *A = ptr(s.a_kind, s.a_inter);
      if (!A) throw std::runtime_error("engine: missing operand");
      if (s.b_kind < 0) {
        gather_axpy(L, s.M, s.alpha, A, s.arow, C, s.crow, size(s.a_kind, s.a_inter), csize);
      } else {
        const double *B = ptr(s.b_kind, s.b_inter);
        if (!B) throw std::runtime_error("engine: missing operand");
        gather_gemm(L, s.M, s.N, s.K, s.alpha, A, s.arow, s.acol, B, s.brow, s.bcol, C, s.crow, s.ccol, true,
                    size(s.a_kind, s.a_inter), size(s.b_kind, s.b_inter), csize);
      }
    }
  }
  if (refresh) cache_version_ = version;
}

}  // namespace fnocc
