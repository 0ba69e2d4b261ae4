// Compiles planned terms (planner.cpp) into offset tables and launches them
// through the gather-GEMM-scatter kernel (kernels.cu).
#include "engine.hpp"

#include <algorithm>
#include <tuple>
#include <functional>
#include <map>
#include <mutex>

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
  copy_now(dev.p, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice);
  std::vector<long long> rk((size_t)std::max(k, 1) * (n + 1), 0);
  for (int i = 0; i < k; ++i)
    for (int x = 1; x <= n; ++x) rk[(size_t)i * (n + 1) + x] = rk[(size_t)i * (n + 1) + x - 1] + binom_ll(n - x, k - 1 - i);
  rankdev.reserve(rk.size() * sizeof(long long));
  copy_now(rankdev.p, rk.data(), rk.size() * sizeof(long long), cudaMemcpyHostToDevice);
}

namespace {

// Storage description of an operand: a list of dimensions, each holding one
// label (plain index) or a packed group of labels stored as sorted tuples.
struct SDim {
  std::vector<int> labels;
  bool packed = false;
  bool positional = false;  // intermediate: indexed by position in the canonical tuple order
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
    d.positional = true;
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

// Canonical tuple order of an index group: tuples (strictly increasing if
// packed) sorted by spin sum (alpha = even index +1, beta = odd -1), then
// lexicographically. Every table, every intermediate dimension and every
// spin segment uses this order.
struct GroupEnum {
  std::vector<int> flat;  // count * k indices
  std::vector<std::tuple<int, long long, long long>> segs;  // (spin sum, start, length)
  long long count = 0;
};

const GroupEnum &enumerate_group(int n, int k, bool packed) {
  // shared by all contexts (host threads): entries are never erased, so the
  // returned references stay valid
  static std::map<std::tuple<int, int, bool>, GroupEnum> cache;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(n, k, packed);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  std::vector<std::vector<int>> tup;
  std::vector<int> cur(k);
  if (packed) {
    for (int j = 0; j < k; ++j) cur[j] = j;
    if (binom_ll(n, k) > 0)
      while (true) {
        tup.push_back(cur);
        int i = k - 1;
        while (i >= 0 && cur[i] == n - k + i) --i;
        if (i < 0) break;
        ++cur[i];
        for (int j = i + 1; j < k; ++j) cur[j] = cur[j - 1] + 1;
      }
  } else {
    long long tot = 1;
    for (int j = 0; j < k; ++j) tot *= n;
    for (long long x = 0; x < tot; ++x) {
      long long rem = x;
      for (int j = k - 1; j >= 0; --j) {
        cur[j] = (int)(rem % n);
        rem /= n;
      }
      tup.push_back(cur);
    }
  }
  auto spin = [](const std::vector<int> &t) {
    int sm = 0;
    for (int x : t) sm += (x % 2 == 0) ? 1 : -1;
    return sm;
  };
  std::stable_sort(tup.begin(), tup.end(),
                   [&](const std::vector<int> &a, const std::vector<int> &b) { return spin(a) < spin(b); });
  GroupEnum ge;
  ge.count = (long long)tup.size();
  for (long long r = 0; r < ge.count; ++r) {
    ge.flat.insert(ge.flat.end(), tup[r].begin(), tup[r].end());
    int sm = spin(tup[r]);
    if (ge.segs.empty() || std::get<0>(ge.segs.back()) != sm) ge.segs.emplace_back(sm, r, 0);
    ++std::get<2>(ge.segs.back());
  }
  return cache.emplace(key, std::move(ge)).first->second;
}

struct TableBuilder {
  std::vector<long long> host;
  struct Pending { DMap *map; std::vector<long long> offs; };
  std::vector<Pending> pend;
  std::map<const DMap *, std::vector<long long>> hoffs;  // host offset of each group's table

  // flat offsets of the rows of `map` restricted to segments (start, length)
  // per group (group ng-1 fastest, as map_off decomposes), appended to out;
  // returns the largest entry
  long long flatten(const DMap &map, const std::vector<std::pair<long long, long long>> &segs,
                    std::vector<long long> &out) const {
    const auto &offs = hoffs.at(&map);
    const int ng = map.ng;
    long long total = 1;
    for (int g = 0; g < ng; ++g) total *= segs[g].second;
    long long mx = 0;
    std::vector<long long> idx(ng, 0);
    for (long long r = 0; r < total; ++r) {
      long long off = 0;
      for (int g = 0; g < ng; ++g) off += host[offs[g] + segs[g].first + idx[g]];
      out.push_back(off);
      mx = std::max(mx, off);
      for (int g = ng - 1; g >= 0; --g) {
        if (++idx[g] < segs[g].second) break;
        idx[g] = 0;
      }
    }
    return mx;
  }

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
      // a packed or intermediate (positional) storage dimension is read only
      // as the same group, by canonical position
      const SDim *whole = nullptr;
      for (auto &d : s.dims)
        if ((d.packed || d.positional) && d.labels == dg.labels) whole = &d;
      const GroupEnum &ge = enumerate_group(n, dg.k, dg.packed && dg.k >= 2);
      if (whole) {
        if (whole->packed != (dg.packed && dg.k >= 2)) throw std::runtime_error("engine: storage packing mismatch");
        for (long long r = 0; r < whole->size; ++r) host.push_back(r * whole->stride);
        cnt = whole->size;
      } else {
        // label by label: every single-label dimension (dense operands and
        // accumulators as well as intermediates) holds the index at its
        // canonical position within its space (the order of the one-index
        // tuple table: one spin block contiguous); the kernels that fill and
        // drain the dense tensors use the same order
        std::vector<long long> st(dg.k), bs(dg.k);
        const GroupEnum &g1 = enumerate_group(n, 1, false);
        std::vector<long long> pos(n, 0);
        for (long long r = 0; r < g1.count; ++r) pos[g1.flat[r]] = r;
        for (int j = 0; j < dg.k; ++j) {
          const SDim *hit = nullptr;
          for (auto &d : s.dims)
            if (!d.packed && d.labels.size() == 1 && d.labels[0] == dg.labels[j]) hit = &d;
          if (!hit) throw std::runtime_error("engine: label not addressable in operand storage");
          st[j] = hit->stride;
          bs[j] = hit->base;
        }
        for (long long r = 0; r < ge.count; ++r) {
          long long off = 0;
          for (int j = 0; j < dg.k; ++j) off += st[j] * (bs[j] + pos[ge.flat[r * dg.k + j]]);
          host.push_back(off);
        }
        cnt = ge.count;
      }
      map->n[g] = cnt;
      long long mx = 0;
      for (long long q = p.offs.back(); q < (long long)host.size(); ++q) mx = std::max(mx, host[q]);
      map->maxoff += mx;
      total *= cnt;
    }
    hoffs[map] = p.offs;
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
    hoffs[map] = p.offs;
    pend.push_back(p);
    return total;
  }

  // device copy (or, for host-only plans, a host copy kept in `keep`)
  void upload(DevBuf &buf, bool host_only, std::vector<long long> &keep) {
    if (host.empty()) host.push_back(0);
    const long long *base;
    if (host_only) {
      keep = host;
      base = keep.data();
    } else {
      buf.reserve(host.size() * sizeof(long long));
      copy_now(buf.p, host.data(), host.size() * sizeof(long long), cudaMemcpyHostToDevice);
      base = buf.as<long long>();
    }
    for (auto &p : pend)
      for (size_t g = 0; g < p.offs.size(); ++g) p.map->tab[g] = base + p.offs[g];
  }
};

}  // namespace

namespace {

// Spin bookkeeping of an operand: the sign each label carries in its charge
// (particle-like / creator +1, hole-like / annihilator -1) and the charge
// sum_labels sign * spin, conserved by every tensor of the method.
struct SpinInfo {
  std::map<int, int> sign;
  int charge = 0;
};

SpinInfo input_spin(const Operand &op, int r_charge) {
  SpinInfo si;
  for (size_t i = 0; i < op.labels.size(); ++i) {
    int sg;
    if (op.kind == TK_F)
      sg = i == 0 ? 1 : -1;
    else if (op.kind == TK_V)
      sg = i < 2 ? 1 : -1;
    else
      sg = lab_space(op.labels[i]) == SP_V ? 1 : -1;
    si.sign[op.labels[i]] = sg;
  }
  si.charge = (op.kind >= TK_R1 && op.kind <= TK_R3) ? r_charge : 0;
  return si;
}

// group sign in an operand, 0 if its labels disagree or are unknown
int group_sign(const DimGroup &g, const SpinInfo &si) {
  int sg = 0;
  for (int l : g.labels) {
    auto it = si.sign.find(l);
    if (it == si.sign.end()) return 0;
    if (sg == 0) sg = it->second;
    if (sg != it->second) return 0;
  }
  return sg;
}

}  // namespace

namespace {
using Segs = std::vector<std::pair<long long, long long>>;
Segs full_segs(const DMap &m) {
  Segs v;
  for (int g = 0; g < m.ng; ++g) v.push_back({0, m.n[g]});
  return v;
}
long long seg_count(const Segs &sg) {
  long long t = 1;
  for (auto &x : sg) t *= x.second;
  return t;
}

// Tasks of a binary step: spin-allowed blocks with equal (row, column)
// segments merge into one task whose reduction runs over all their K
// segments in turn. Flat tables go to flat_host (row and column tables shared
// between tasks).
void build_tasks(const TableBuilder &tb, ExecStep &e, std::vector<long long> &flat_host) {
  std::map<std::pair<Segs, Segs>, std::vector<Segs>> by_mn;
  if (e.blocked) {
    for (const SubGemm &b : e.blocks)
      if (b.M > 0 && b.N > 0 && b.K > 0) by_mn[{b.mseg, b.nseg}].push_back(b.kseg);
  } else {
    by_mn[{full_segs(e.arow), full_segs(e.bcol)}].push_back(full_segs(e.acol));
  }
  std::map<std::pair<const DMap *, Segs>, std::pair<long long, long long>> memo;  // -> (offset, max)
  auto flat = [&](const DMap &m, const Segs &sg) {
    auto key = std::make_pair(&m, sg);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    long long off = (long long)flat_host.size();
    long long mx = tb.flatten(m, sg, flat_host);
    return memo[key] = {off, mx};
  };
  e.grouped = true;
  for (auto &kv : by_mn) {
    ExecStep::TaskRef tr;
    auto ar = flat(e.arow, kv.first.first), cr = flat(e.crow, kv.first.first);
    auto bc = flat(e.bcol, kv.first.second), cc = flat(e.ccol, kv.first.second);
    tr.acol = (long long)flat_host.size();
    long long amx = 0, bmx = 0;
    for (auto &ks : kv.second) amx = std::max(amx, tb.flatten(e.acol, ks, flat_host));
    tr.brow = (long long)flat_host.size();
    for (auto &ks : kv.second) bmx = std::max(bmx, tb.flatten(e.brow, ks, flat_host));
    tr.K = tr.brow - tr.acol;
    tr.M = seg_count(kv.first.first);
    tr.N = seg_count(kv.first.second);
    if (tr.M == 0 || tr.N == 0 || tr.K == 0) continue;  // contributes nothing
    tr.arow = ar.first;
    tr.crow = cr.first;
    tr.bcol = bc.first;
    tr.ccol = cc.first;
    e.gmax_a = std::max(e.gmax_a, ar.second + amx);
    e.gmax_b = std::max(e.gmax_b, bmx + bc.second);
    e.gmax_c = std::max(e.gmax_c, cr.second + cc.second);
    e.tasks.push_back(tr);
  }
}

}  // namespace

ExecEquation::ExecEquation(const Equation &eq, int o, int v, const int rdims[3][2], double amortize,
                           double cache_cap, int r_charge, bool host_only, int sms)
    : nh_(eq.nh), np_(eq.np), o_(o), v_(v), sms_(sms > 0 ? sms : 152), host_only_(host_only) {
  TableBuilder tb;
  std::vector<long long> flat_host;
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
    std::vector<SpinInfo> inter_spin(plan.inter_dims.size());
    std::vector<char> inter_spin_set(plan.inter_dims.size(), 0);
    auto spin_of = [&](const Operand &op) -> SpinInfo {
      if (op.kind == TK_INTERMEDIATE) return inter_spin.at(op.inter);
      return input_spin(op, r_charge);
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
      const bool binary = s.b.kind >= 0;
      if (binary) {
        Storage sb = storage_of(s.b);
        e.K = tb.add(&e.acol, s.kg, sa, o, v);
        tb.add(&e.brow, s.kg, sb, o, v);
        e.N = tb.add(&e.bcol, s.ng, sb, o, v);
        if (s.to_output)
          tb.add(&e.ccol, s.ng, sc, o, v);
        else
          tb.add_positional(&e.ccol, s.ng, sc, (int)s.mg.size());
      } else {
        e.N = 1;
        e.K = 1;
      }
      // spin: charges and group signs; the result's spin info for intermediates
      SpinInfo sa_spin = spin_of(s.a), sb_spin;
      if (binary) sb_spin = spin_of(s.b);
      if (!s.to_output && !inter_spin_set[s.out_inter]) {
        // the producer writes the intermediate's dims positionally (mg, then ng):
        // dim d takes the signs of the producer's group d
        SpinInfo r;
        const auto &dims = plan.inter_dims.at(s.out_inter);
        size_t d = 0;
        for (int side = 0; side < 2; ++side) {
          const auto &gs = side == 0 ? s.mg : s.ng;
          const SpinInfo &src = side == 0 ? sa_spin : sb_spin;
          for (auto &g : gs) {
            if (d >= dims.size() || dims[d].labels.size() != g.labels.size())
              throw std::runtime_error("engine: producer groups do not match the intermediate");
            for (size_t j = 0; j < g.labels.size(); ++j) {
              auto it = src.sign.find(g.labels[j]);
              r.sign[dims[d].labels[j]] = it == src.sign.end() ? 0 : it->second;
            }
            ++d;
          }
        }
        r.charge = sa_spin.charge + (binary ? sb_spin.charge : 0);
        inter_spin[s.out_inter] = r;
        inter_spin_set[s.out_inter] = 1;
      }
      // spin-allowed sub-GEMMs of large steps
      const double full = binary ? 2.0 * double(e.M) * double(e.N) * double(e.K) : double(e.M);
      std::vector<const DimGroup *> groups;
      std::vector<int> sig_a, sig_b;
      for (auto &g : s.mg) {
        groups.push_back(&g);
        sig_a.push_back(group_sign(g, sa_spin));
        sig_b.push_back(0);
      }
      if (binary) {
        for (auto &g : s.kg) {
          groups.push_back(&g);
          sig_a.push_back(group_sign(g, sa_spin));
          sig_b.push_back(group_sign(g, sb_spin));
        }
        for (auto &g : s.ng) {
          groups.push_back(&g);
          sig_a.push_back(0);
          sig_b.push_back(group_sign(g, sb_spin));
        }
      }
      bool signs_ok = true;
      for (size_t gi = 0; gi < groups.size(); ++gi) {
        bool in_a = gi < s.mg.size() + (binary ? s.kg.size() : 0);
        bool in_b = binary && gi >= s.mg.size();
        if ((in_a && sig_a[gi] == 0) || (in_b && sig_b[gi] == 0)) signs_ok = false;
      }
      double done_flops = full;
      if (signs_ok && full >= 1e7) {
        std::vector<const GroupEnum *> ge;
        for (auto *g : groups) ge.push_back(&enumerate_group(g->space == SP_O ? o : v, g->k, g->packed && g->k >= 2));
        std::vector<int> pick(groups.size(), 0);
        const size_t nm = s.mg.size(), nk = binary ? s.kg.size() : 0;
        double blocked_flops = 0;
        std::function<void(size_t, int, int)> rec = [&](size_t gi, int ca, int cb) {
          if (gi == groups.size()) {
            if (ca != sa_spin.charge) return;
            if (binary && cb != sb_spin.charge) return;
            SubGemm b;
            b.M = b.N = b.K = 1;
            for (size_t q = 0; q < groups.size(); ++q) {
              auto &sg = ge[q]->segs[pick[q]];
              std::pair<long long, long long> seg(std::get<1>(sg), std::get<2>(sg));
              if (q < nm) {
                b.mseg.push_back(seg);
                b.M *= seg.second;
              } else if (q < nm + nk) {
                b.kseg.push_back(seg);
                b.K *= seg.second;
              } else {
                b.nseg.push_back(seg);
                b.N *= seg.second;
              }
            }
            blocked_flops += binary ? 2.0 * double(b.M) * double(b.N) * double(b.K) : double(b.M);
            e.blocks.push_back(b);
            return;
          }
          for (size_t k = 0; k < ge[gi]->segs.size(); ++k) {
            pick[gi] = (int)k;
            int sv = std::get<0>(ge[gi]->segs[k]);
            rec(gi + 1, ca + sig_a[gi] * sv, cb + sig_b[gi] * sv);
          }
        };
        rec(0, 0, 0);
        e.blocked = true;
        done_flops = blocked_flops;
      }
      (s.constant ? cached_flops_ : flops_) += done_flops;
      if (binary && double(e.M) * double(e.N) > 256.0) build_tasks(tb, e, flat_host);
    }
    terms_.push_back(std::move(et));
  }
  (void)rdims;
  tb.upload(tables_, host_only_, host_tables_);
  build_launches(flat_host);
}

// Uploads the flat tables, then builds for every grouped step and tile shape
// its GTask array: tiles, a split of the reduction when the step has few
// tiles, CTA, partial and reduction offsets.
//
// FP64 tiles are FMA-bound and several CTAs share an SM's FP64 pipe, so a
// launch of c roughly equal CTAs that are all resident at once takes about
// ceil(c / 152) CTA-times. The reduction split of the FP64 shapes starts
// from two CTAs per SM and grows, up to about four per SM, while that lowers
// ceil(c / 152) / c by more than 1 %; the shape estimate carries the same
// factor.
void ExecEquation::build_launches(const std::vector<long long> &flat_host) {
  if (flat_host.empty()) return;
  const long long *fb;
  if (host_only_) {
    host_flat_ = flat_host;
    fb = host_flat_.data();
  } else {
    flat_.reserve(sizeof(long long) * flat_host.size());
    copy_now(flat_.p, flat_host.data(), sizeof(long long) * flat_host.size(), cudaMemcpyHostToDevice);
    fb = flat_.as<long long>();
  }
  const long long kSms = std::max(1, sms_);
  const long long kWantCta = 2 * kSms;   // at least two CTAs per SM where the tiles allow
  const long long kFillCta = 4 * kSms;   // FP64 shapes: split at most up to four CTAs per SM
  constexpr long long kPartCap = 1LL << 27;  // doubles of split partials per launch
  constexpr long long kPanelCap = kPanelCapBytes;
  // CTA-times per CTA of a launch of c equal resident CTAs (smaller is better)
  auto wave_cost = [kSms](long long c) { return double((c + kSms - 1) / kSms) / double(std::max<long long>(1, c)); };
  std::vector<GTask> gt;
  std::vector<int> sid;
  struct Fix { GroupedLaunch *gl; size_t t0, s0; };
  std::vector<Fix> fix;
  for (ExecTerm &t : terms_)
    for (ExecStep &e : t.steps) {
      if (!e.grouped) continue;
      double est[kGShapesAll];
      for (int shape = 0; shape < kGShapesAll; ++shape) {
        int tbm, tbn, tbk;
        grouped_shape(shape, &tbm, &tbn, &tbk);
        long long T = 0;
        for (auto &tr : e.tasks) T += ((tr.M + tbm - 1) / tbm) * ((tr.N + tbn - 1) / tbn);
        // at least two CTAs per SM where the tiles allow it (one CTA's
        // gathers overlap another's multiply-adds)
        T = std::max<long long>(T, 1);
        long long want = T < kWantCta ? (kWantCta + T - 1) / T : 1;
        if (shape < kGShapeBf16 && T < kFillCta) {
          const long long wmax = (kFillCta + T - 1) / T;
          for (long long w = want + 1; w <= wmax; ++w)
            if (wave_cost(T * w) < 0.99 * wave_cost(T * want)) want = w;
        }
        GroupedLaunch &gl = e.gl[shape];
        gl.shape = shape;
        gl.ntasks = (int)e.tasks.size();
        fix.push_back({&gl, gt.size(), sid.size()});
        long long cta = 0, part = 0, red = 0, pk_blocks = 0, pbytes = 0;
        long long pa_bytes = 0, pb_bytes = 0;
        if (shape_kind(shape) == 3) tcp_block_bytes(shape - kGShapeTcp, &pa_bytes, &pb_bytes);
        double padded = 0, flops = 0;
        for (size_t i = 0; i < e.tasks.size(); ++i) {
          const auto &tr = e.tasks[i];
          GTask g;
          g.M = tr.M;
          g.N = tr.N;
          g.K = tr.K;
          g.arow = fb + tr.arow;
          g.acol = fb + tr.acol;
          g.brow = fb + tr.brow;
          g.bcol = fb + tr.bcol;
          g.crow = fb + tr.crow;
          g.ccol = fb + tr.ccol;
          const long long tm = (tr.M + tbm - 1) / tbm;
          g.tiles_n = (tr.N + tbn - 1) / tbn;
          g.tiles = tm * g.tiles_n;
          // reduction chunks of at least 4 K tiles (FP64) or 2 (tensor-core
          // tiles, whose K tile is cheap next to the launch's CTA count)
          const long long min_tiles = shape < kGShapeBf16 ? 4 : 2;
          long long ks = std::min<long long>(want, std::max<long long>(1, tr.K / (min_tiles * tbk)));
          if (ks > 1 && part + ks * tr.M * tr.N > kPartCap) ks = 1;
          long long kchunk = (tr.K + ks - 1) / ks;
          kchunk = (kchunk + tbk - 1) / tbk * tbk;
          ks = (tr.K + kchunk - 1) / kchunk;
          g.ksplit = (int)ks;
          g.kchunk = kchunk;
          g.mfast = tr.N > tr.M ? 1 : 0;
          if (shape_kind(shape) == 3) {
            // split BF16 panels of the whole K range of the task, 256-byte aligned
            g.ksteps = (int)((tr.K + 15) / 16);
            g.apanel = pbytes;
            pbytes += (tm * g.ksteps * pa_bytes + 255) / 256 * 256;
            g.bpanel = pbytes;
            pbytes += (g.tiles_n * g.ksteps * pb_bytes + 255) / 256 * 256;
            g.pk_begin = pk_blocks;
            pk_blocks += (tm + g.tiles_n) * g.ksteps;
          }
          g.cta_begin = cta;
          cta += g.tiles * ks;
          if (ks > 1) {
            g.part_off = part;
            part += ks * tr.M * tr.N;
            g.red_begin = red;
            red += tr.M * tr.N;
            sid.push_back((int)i);
          }
          padded += 2.0 * double(tm * tbm) * double(g.tiles_n * tbn) * double((tr.K + tbk - 1) / tbk * tbk);
          flops += 2.0 * double(tr.M) * double(tr.N) * double(tr.K);
          gt.push_back(g);
        }
        if (cta > 0x7fffffffLL) throw std::runtime_error("engine: grouped grid too large");
        gl.ncta = cta;
        gl.nsplit = (int)(sid.size() - fix.back().s0);
        gl.nred = red;
        gl.part_need = part;
        gl.padded = padded;
        gl.flops = flops;
        gl.pack_blocks = pk_blocks;
        gl.panel_bytes = pbytes;
        if (shape_kind(shape) == 3) {
          // panel tiles: chosen by timing only (large steps), or when forced;
          // here ranked by padded work, excluded above the panel memory cap
          est[shape] = pbytes <= kPanelCap ? padded : 1e300;
        } else if (shape < kGShapeBf16) {
          est[shape] = padded * wave_cost(cta);
        } else {
          // tensor-core tiles: the cost is staging (gather, convert, split) of
          // the (tbm + tbn) x tbk operand panels of every K tile, over the
          // CTAs resident at once (two per SM; one for the 128 x 256 tcgen05
          // tile, whose stages take 145 KiB of shared memory)
          double staged = 0;
          for (size_t i = gt.size() - e.tasks.size(); i < gt.size(); ++i)
            staged += double(gt[i].tiles) * double((gt[i].K + tbk - 1) / tbk) * double((tbm + tbn) * tbk);
          const long long per_sm = (shape_kind(shape) == 2 && tbn >= 256) ? 1 : 2;
          est[shape] = staged / double(std::max<long long>(1, std::min<long long>(cta, per_sm * kSms)));
        }
      }
      int bbest = kGShapeBf16;
      for (int shape = kGShapeBf16 + 1; shape < kGShapeTc; ++shape)
        if (est[shape] < est[bbest]) bbest = shape;
      e.bf16_shape = bbest;
      // gathering tcgen05 tiles: the best with the rows of A on the
      // accumulator lanes (the first three) and the best transposed one
      int tbest = kGShapeTc, tbest_t = kGShapeTc + 3;
      for (int shape = kGShapeTc + 1; shape < kGShapeTc + 3; ++shape)
        if (est[shape] < est[tbest]) tbest = shape;
      for (int shape = kGShapeTc + 4; shape < kGShapeTcp; ++shape)
        if (est[shape] < est[tbest_t]) tbest_t = shape;
      e.tc_shape = est[tbest_t] < est[tbest] ? tbest_t : tbest;
      e.tc_shape_alt = est[tbest_t] < est[tbest] ? tbest : tbest_t;
      int pbest = kGShapeTcp;
      for (int shape = kGShapeTcp + 1; shape < kGShapesAll; ++shape)
        if (est[shape] < est[pbest]) pbest = shape;
      e.tcp_shape = est[pbest] < 1e300 ? pbest : -1;
      // BF16x3: the tcgen05 tile where it stages less per busy SM (large
      // steps time both once, see run)
      e.bf16x3_shape = est[tbest] < est[bbest] ? tbest : bbest;
      int best = 0;
      for (int shape = 1; shape < kGShapes; ++shape)
        if (est[shape] < est[best]) best = shape;
      e.default_shape = best;
      std::vector<int> order;
      for (int shape = 0; shape < kGShapes; ++shape)
        if (est[shape] <= 1.25 * est[best]) order.push_back(shape);
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return est[a] < est[b]; });
      if (order.size() > 4) order.resize(4);
      e.cand = order;
    }
  const size_t tbytes = sizeof(GTask) * gt.size(), ibytes = sizeof(int) * sid.size();
  const size_t ioff = (tbytes + 255) / 256 * 256;
  const GTask *tb;
  const int *ib;
  if (host_only_) {
    host_gt_ = gt;
    host_sid_ = sid;
    if (host_sid_.empty()) host_sid_.push_back(0);
    tb = host_gt_.data();
    ib = host_sid_.data();
  } else {
    gtasks_.reserve(ioff + std::max<size_t>(ibytes, 8));
    copy_now(gtasks_.p, gt.data(), tbytes, cudaMemcpyHostToDevice);
    if (ibytes) copy_now((char *)gtasks_.p + ioff, sid.data(), ibytes, cudaMemcpyHostToDevice);
    tb = reinterpret_cast<const GTask *>(gtasks_.p);
    ib = reinterpret_cast<const int *>((char *)gtasks_.p + ioff);
  }
  for (auto &f : fix) {
    f.gl->tasks = tb + f.t0;
    f.gl->split_ids = ib + f.s0;
  }
}

bool ExecEquation::autotune = true;

ExecEquation::~ExecEquation() {
  for (auto ev : tune_events_) cudaEventDestroy(ev);
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
      auto sub_map = [](const DMap &full, const std::vector<std::pair<long long, long long>> &seg) {
        DMap m = full;
        for (size_t g = 0; g < seg.size(); ++g) {
          m.tab[g] = full.tab[g] + seg[g].first;
          m.n[g] = seg[g].second;
        }
        return m;
      };
      if (s.blocked && s.b_kind < 0) {  // unary step: spin-allowed blocks only
        for (const SubGemm &b : s.blocks) {
          if (b.M == 0) continue;
          DMap arow = sub_map(s.arow, b.mseg), crow = sub_map(s.crow, b.mseg);
          gather_axpy(L, b.M, s.alpha, A, arow, C, crow, size(s.a_kind, s.a_inter), csize);
        }
        continue;
      }
      if (s.b_kind < 0) {
        gather_axpy(L, s.M, s.alpha, A, s.arow, C, s.crow, size(s.a_kind, s.a_inter), csize);
        continue;
      }
      const double *B = ptr(s.b_kind, s.b_inter);
      if (!B) throw std::runtime_error("engine: missing operand");
      if (!s.grouped) {  // output of at most 256 elements: the small-output kernel
        gather_gemm(L, s.M, s.N, s.K, s.alpha, A, s.arow, s.acol, B, s.brow, s.bcol, C, s.crow, s.ccol, true,
                    size(s.a_kind, s.a_inter), size(s.b_kind, s.b_inter), csize);
        continue;
      }
      if (s.gmax_a >= size(s.a_kind, s.a_inter) || s.gmax_b >= size(s.b_kind, s.b_inter) || s.gmax_c >= csize)
        throw std::runtime_error("engine: grouped index tables exceed operand bounds");
      ExecStep &ms = const_cast<ExecStep &>(s);
      if (L.precision != 0 && s.gl[0].flops >= 1e5) {
        // split products: mma.sync tiles for TF32x3; for BF16x3 the mma.sync
        // or the tcgen05 tile, timed once for large steps
        ExecStep &mm = const_cast<ExecStep &>(s);
        const int fk = L.force_shape >= 0 && L.force_shape < kGShapesAll ? shape_kind(L.force_shape) : 0;
        int shape;
        if (fk == 1 || ((fk == 2 || fk == 3) && L.precision == 1))
          shape = L.force_shape;
        else if (L.precision != 1)
          shape = s.bf16_shape;
        else if (mm.tuned_mixed >= 0)
          shape = mm.tuned_mixed;
        else if (autotune && s.gl[s.bf16x3_shape].padded >= 1e8) {
          // the mma.sync and gathering tcgen05 tiles of least staged volume,
          // and every panel tile within the panel memory cap
          std::vector<int> cand = {s.bf16_shape, s.tc_shape, s.tc_shape_alt};
          for (int k = kGShapeTcp; k < kGShapesAll; ++k)
            if (s.gl[k].panel_bytes <= kPanelCapBytes) cand.push_back(k);
          tune_launch(L, mm.mixed_tune, cand, mm.tuned_mixed, s, A, B, C);
          continue;
        } else
          shape = s.bf16x3_shape;
        grouped_gemm(L, s.gl[shape], s.alpha, A, B, C);
        continue;
      }
      if (L.precision == 0 && L.force_shape >= 0 && L.force_shape < kGShapes) {
        grouped_gemm(L, s.gl[L.force_shape], s.alpha, A, B, C);
        continue;
      }
      const bool tune = autotune && L.precision == 0 && ms.tuned_shape < 0 && ms.cand.size() > 1 &&
                        s.gl[s.default_shape].padded >= 1e8;
      if (!tune) {
        grouped_gemm(L, s.gl[ms.tuned_shape >= 0 ? ms.tuned_shape : s.default_shape], s.alpha, A, B, C);
        continue;
      }
      if (ms.pending < 0) {  // first use: an event pair of its own
        ms.pending = tune_count_++;
        while ((int)tune_events_.size() < 2 * tune_count_) {
          cudaEvent_t ev;
          FNOCC_CUDA(cudaEventCreate(&ev));
          tune_events_.push_back(ev);
        }
      }
      cudaEvent_t e0 = tune_events_[2 * ms.pending], e1 = tune_events_[2 * ms.pending + 1];
      for (int k : ms.cand)
        if (ms.trial_ms[k] < 0) {  // the trial of the previous run
          FNOCC_CUDA(cudaEventSynchronize(e1));
          float tms = 0;
          FNOCC_CUDA(cudaEventElapsedTime(&tms, e0, e1));
          ms.trial_ms[k] = std::max(tms, 1e-6f);
        }
      int next = -1;
      for (int k : ms.cand)
        if (next < 0 && ms.trial_ms[k] == 0) next = k;
      if (next < 0) {
        int best = ms.cand[0];
        for (int k : ms.cand)
          if (ms.trial_ms[k] < ms.trial_ms[best]) best = k;
        ms.tuned_shape = best;
        grouped_gemm(L, s.gl[best], s.alpha, A, B, C);
        continue;
      }
      FNOCC_CUDA(cudaEventRecord(e0, L.stream));
      grouped_gemm(L, s.gl[next], s.alpha, A, B, C);
      FNOCC_CUDA(cudaEventRecord(e1, L.stream));
      ms.trial_ms[next] = -1.f;  // in flight; read on the next run
    }
  }
  if (refresh) cache_version_ = version;
}

bool ExecEquation::tuning_pending(const Launch &L) const {
  if (!autotune || L.force_shape >= 0) return false;
  for (const ExecTerm &t : terms_)
    for (const ExecStep &s : t.steps) {
      // cached R-independent steps do not run while the cache is valid
      if (!s.grouped || s.b_kind < 0 || s.constant) continue;
      if (L.precision == 0) {
        if (s.tuned_shape < 0 && s.cand.size() > 1 && s.gl[s.default_shape].padded >= 1e8) return true;
      } else if (L.precision == 1 && s.gl[0].flops >= 1e5) {
        if (s.tuned_mixed < 0 && s.gl[s.bf16x3_shape].padded >= 1e8) return true;
      }
    }
  return false;
}

void ExecEquation::tune_launch(const Launch &L, ExecStep::Trial &tr, const std::vector<int> &cand, int &tuned,
                               const ExecStep &s, const double *A, const double *B, double *C) {
  if (tr.pending < 0) {  // first use: an event pair of its own
    tr.pending = tune_count_++;
    while ((int)tune_events_.size() < 2 * tune_count_) {
      cudaEvent_t ev;
      FNOCC_CUDA(cudaEventCreate(&ev));
      tune_events_.push_back(ev);
    }
  }
  cudaEvent_t e0 = tune_events_[2 * tr.pending], e1 = tune_events_[2 * tr.pending + 1];
  for (int k : cand)
    if (tr.ms[k] < 0) {  // the trial of the previous run
      FNOCC_CUDA(cudaEventSynchronize(e1));
      float tms = 0;
      FNOCC_CUDA(cudaEventElapsedTime(&tms, e0, e1));
      tr.ms[k] = std::max(tms, 1e-6f);
    }
  int next = -1;
  for (int k : cand)
    if (next < 0 && tr.ms[k] == 0) next = k;
  if (next < 0) {
    int best = cand.front();
    for (int k : cand)
      if (tr.ms[k] < tr.ms[best]) best = k;
    tuned = best;
    grouped_gemm(L, s.gl[best], s.alpha, A, B, C);
    return;
  }
  FNOCC_CUDA(cudaEventRecord(e0, L.stream));
  grouped_gemm(L, s.gl[next], s.alpha, A, B, C);
  FNOCC_CUDA(cudaEventRecord(e1, L.stream));
  tr.ms[next] = -1.f;  // in flight; read on the next run
}

namespace {
long long host_map_off(const DMap &mp, long long m) {
  long long off = 0;
  for (int g = mp.ng - 1; g >= 0; --g) {
    const long long q = m / mp.n[g];
    off += mp.tab[g][m - q * mp.n[g]];
    m = q;
  }
  return off;
}
DMap host_sub(const DMap &full, const std::vector<std::pair<long long, long long>> &seg) {
  DMap m = full;
  for (size_t g = 0; g < seg.size(); ++g) {
    m.tab[g] = full.tab[g] + seg[g].first;
    m.n[g] = seg[g].second;
  }
  return m;
}
}  // namespace

// Every grouped step of a host-only plan: the (A, B, C) element-offset
// triples its tasks address, for every tile shape's task list, against the
// triples of the spin-allowed blocks decoded through the per-group tables.
void ExecEquation::stats(double out[10]) const {
  // model time of one launch on the FP64 pipe: padded multiply-adds of its
  // busiest SM, ceil(c / sms) CTA-times of padded / c each, at 2 FMA per
  // clock per SM and 2.07 GHz
  constexpr double kSmFlops = 2.0 * 2.0 * 2.07e9;
  for (int k = 0; k < 10; ++k) out[k] = 0;
  out[8] = double(scratch_need_);
  out[9] = double(cache_need_);
  for (const ExecTerm &t : terms_)
    for (const ExecStep &e : t.steps) {
      if (e.constant) continue;  // cached: once per H-bar, not per product
      if (!e.grouped) {
        out[6] += 1;
        out[7] += 2.0 * double(e.M) * double(e.N) * double(e.K);
        continue;
      }
      const GroupedLaunch &g = e.gl[e.default_shape];
      const double c = double(std::max<long long>(1, g.ncta));
      const double waves = std::ceil(c / double(sms_));
      out[0] += 1;
      out[1] += g.flops;
      out[2] += g.padded;
      out[3] += g.padded * waves / c / kSmFlops;
      if (g.ncta < sms_) {
        out[4] += 1;
        out[5] += g.flops;
      }
    }
}

long long ExecEquation::self_check(double max_work) const {
  if (!host_only_) throw std::runtime_error("self_check needs a host-only plan");
  long long bad = 0;
  using Trip = std::tuple<long long, long long, long long>;
  for (const ExecTerm &t : terms_)
    for (const ExecStep &s : t.steps) {
      if (!s.grouped) continue;
      double work = 0;
      for (auto &tr : s.tasks) work += double(tr.M) * double(tr.N) * double(tr.K);
      // launch descriptors of every shape: checked for every step
      for (int shape = 0; shape < kGShapesAll; ++shape) {
        const GroupedLaunch &gl = s.gl[shape];
        int tbm, tbn, tbk;
        grouped_shape(shape, &tbm, &tbn, &tbk);
        long long ctas = 0, part = 0, red = 0;
        int nsplit = 0;
        for (int i = 0; i < gl.ntasks; ++i) {
          const GTask &g = gl.tasks[i];
          if (g.cta_begin != ctas) ++bad;  // CTA ranges must tile the grid in order
          ctas += g.tiles * g.ksplit;
          if ((long long)g.ksplit * g.kchunk < g.K) ++bad;  // the splits cover K
          if (g.ksplit > 1 && (long long)(g.ksplit - 1) * g.kchunk >= g.K) ++bad;  // no empty split
          if (g.kchunk % tbk != 0) ++bad;  // whole K tiles per split
          // the kernel's tiling of this shape
          if (g.tiles_n != (g.N + tbn - 1) / tbn || g.tiles != ((g.M + tbm - 1) / tbm) * g.tiles_n) ++bad;
          if (g.ksplit > 1) {  // partial sums and their ordered reduction tile their buffers in order
            ++nsplit;
            if (g.part_off != part || g.red_begin != red) ++bad;
            part += (long long)g.ksplit * g.M * g.N;
            red += g.M * g.N;
          }
        }
        if (ctas != gl.ncta) ++bad;
        if (part != gl.part_need || red != gl.nred || nsplit != gl.nsplit) ++bad;
      }
      if (work > max_work) continue;
      std::vector<Trip> ref;
      auto add_ref = [&](long long M, long long N, long long K, const DMap &ar, const DMap &ac, const DMap &br,
                         const DMap &bc, const DMap &cr, const DMap &cc) {
        for (long long m = 0; m < M; ++m)
          for (long long n = 0; n < N; ++n)
            for (long long k = 0; k < K; ++k)
              ref.emplace_back(host_map_off(ar, m) + host_map_off(ac, k), host_map_off(br, k) + host_map_off(bc, n),
                               host_map_off(cr, m) + host_map_off(cc, n));
      };
      if (s.blocked) {
        for (const SubGemm &b : s.blocks)
          if (b.M > 0 && b.N > 0 && b.K > 0)
            add_ref(b.M, b.N, b.K, host_sub(s.arow, b.mseg), host_sub(s.acol, b.kseg), host_sub(s.brow, b.kseg),
                    host_sub(s.bcol, b.nseg), host_sub(s.crow, b.mseg), host_sub(s.ccol, b.nseg));
      } else {
        add_ref(s.M, s.N, s.K, s.arow, s.acol, s.brow, s.bcol, s.crow, s.ccol);
      }
      std::sort(ref.begin(), ref.end());
      for (int shape = 0; shape < kGShapesAll; ++shape) {
        const GroupedLaunch &gl = s.gl[shape];
        std::vector<Trip> got;
        for (int i = 0; i < gl.ntasks; ++i) {
          const GTask &g = gl.tasks[i];
          for (long long m = 0; m < g.M; ++m)
            for (long long n = 0; n < g.N; ++n)
              for (long long k = 0; k < g.K; ++k)
                got.emplace_back(g.arow[m] + g.acol[k], g.brow[k] + g.bcol[n], g.crow[m] + g.ccol[n]);
        }
        std::sort(got.begin(), got.end());
        if (got != ref) ++bad;
      }
    }
  return bad;
}

}  // namespace fnocc
