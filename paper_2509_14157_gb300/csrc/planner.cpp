// Symbolic planner (see planner.hpp). Pure host C++.
//
// Derivation: for a projection <mu| H~ X_1 .. X_n |0> every full contraction
// of the normal-ordered operator strings is enumerated (a quasi-particle
// creator is paired with a quasi-particle annihilator to its left that belongs
// to another string). The value of a contraction is the parity of the
// permutation that brings each pair next to each other times the product of
// the string prefactors. Terms in which H~ is not joined to every X_k are
// dropped (linked form of Eq. 6 and of (H-bar R)_c in Eq. 1-4).
//
// Reduction: terms are brought to a canonical form (tensor order, slot order
// inside antisymmetric groups, dummy names) and summed; terms that differ only
// by a permutation of the projection's holes or particles are collected into
// one orbit, represented once with coefficient c / |stabiliser|; the caller
// applies the full antisymmetriser over the output groups afterwards.
#include "planner.hpp"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <functional>
#include <map>
#include <numeric>
#include <set>
#include <sstream>
#include <stdexcept>

namespace fnocc {

static long long gcdll(long long a, long long b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b) { long long t = a % b; a = b; b = t; }
  return a ? a : 1;
}

Frac::Frac(long long a, long long b) : n(a), d(b) {
  if (d < 0) { n = -n; d = -d; }
  long long g = gcdll(n, d);
  n /= g; d /= g;
}
Frac Frac::operator+(const Frac &o) const { return Frac(n * o.d + o.n * d, d * o.d); }
Frac Frac::operator*(const Frac &o) const { return Frac(n * o.n, d * o.d); }

namespace {

long long factorial(int k) { long long r = 1; for (int i = 2; i <= k; ++i) r *= i; return r; }

// ---- operator strings --------------------------------------------------------

struct OpDef { int space; bool dag; int slot; };

struct StringDef {
  int kind;
  std::vector<OpDef> ops;                 // left to right
  std::vector<std::vector<int>> groups;   // slot groups
  Frac pref;
};

StringDef fock_string(int ps, int qs) {
  return {TK_F, {{ps, true, 0}, {qs, false, 1}}, {{0}, {1}}, Frac(1)};
}

StringDef two_body_string(int p, int q, int r, int s) {
  // 1/4 <pq||rs> {p+ q+ s r}
  return {TK_V, {{p, true, 0}, {q, true, 1}, {s, false, 3}, {r, false, 2}}, {{0, 1}, {2, 3}}, Frac(1, 4)};
}

// nh holes (slots 0..nh-1), np particles (slots nh..): a1+ .. anp+ i_nh .. i1
StringDef excitation_string(int kind, int nh, int np) {
  StringDef s;
  s.kind = kind;
  for (int k = 0; k < np; ++k) s.ops.push_back({SP_V, true, nh + k});
  for (int k = nh - 1; k >= 0; --k) s.ops.push_back({SP_O, false, k});
  std::vector<int> h, p;
  for (int k = 0; k < nh; ++k) h.push_back(k);
  for (int k = 0; k < np; ++k) p.push_back(nh + k);
  s.groups = {h, p};
  s.pref = Frac(1, factorial(nh) * factorial(np));
  return s;
}

std::vector<StringDef> hamiltonian_strings() {
  std::vector<StringDef> out;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) out.push_back(fock_string(a, b));
  for (int m = 0; m < 16; ++m)
    out.push_back(two_body_string((m >> 3) & 1, (m >> 2) & 1, (m >> 1) & 1, m & 1));
  return out;
}

struct SeqOp { int owner; int space; bool dag; int tag; };  // owner -1: projection

bool qp_annihilator(const SeqOp &x) { return (x.space == SP_O) == x.dag; }

// ---- canonical form -------------------------------------------------------------

struct Canon {
  std::vector<int> code;
  int sign;
};

int perm_parity(const std::vector<int> &p) {
  // parity by inversion count
  int inv = 0;
  for (size_t i = 0; i < p.size(); ++i)
    for (size_t j = i + 1; j < p.size(); ++j)
      if (p[i] > p[j]) ++inv;
  return (inv & 1) ? -1 : 1;
}

bool is_external(int lab) { return (lab >> 1) < 64; }

Canon canonical_fixed(std::vector<Factor> fs) {
  // where does each label sit: (factor, group)
  std::map<int, std::vector<std::pair<int, int>>> where;
  for (int fi = 0; fi < (int)fs.size(); ++fi)
    for (int gi = 0; gi < (int)fs[fi].groups.size(); ++gi)
      for (int lab : fs[fi].groups[gi]) where[lab].push_back({fi, gi});
  auto partner = [&](int lab, int fi, int gi) -> std::pair<int, int> {
    const auto &w = where[lab];
    if (w.size() < 2) return {-1, -1};
    return (w[0].first == fi && w[0].second == gi) ? w[1] : w[0];
  };
  // slot key: externals first (by label), then by partner (factor, group)
  auto key = [&](int lab, int fi, int gi) -> long long {
    if (is_external(lab)) return (long long)lab;
    auto p = partner(lab, fi, gi);
    return 1000000LL + p.first * 1000 + p.second;
  };
  int sign = 1;
  for (int fi = 0; fi < (int)fs.size(); ++fi)
    for (auto &g : fs[fi].groups) {
      std::vector<int> idx(g.size());
      std::iota(idx.begin(), idx.end(), 0);
      int gi = int(&g - &fs[fi].groups[0]);
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return key(g[x], fi, gi) < key(g[y], fi, gi); });
      sign *= perm_parity(idx);
      std::vector<int> ng(g.size());
      for (size_t k = 0; k < idx.size(); ++k) ng[k] = g[idx[k]];
      g = ng;
    }
  // align ties: slots of a later group joined to this group follow this group's order
  for (int fi = 0; fi < (int)fs.size(); ++fi)
    for (int gi = 0; gi < (int)fs[fi].groups.size(); ++gi) {
      const auto g = fs[fi].groups[gi];
      std::vector<std::pair<int, int>> targets;
      for (int lab : g) {
        if (is_external(lab)) continue;
        auto p = partner(lab, fi, gi);
        if (p.first > fi && std::find(targets.begin(), targets.end(), p) == targets.end()) targets.push_back(p);
      }
      for (auto tg : targets) {
        std::vector<int> want;
        for (int lab : g)
          if (!is_external(lab) && partner(lab, fi, gi) == tg) want.push_back(lab);
        auto &h = fs[tg.first].groups[tg.second];
        std::vector<int> pos;
        for (int p = 0; p < (int)h.size(); ++p)
          if (std::find(want.begin(), want.end(), h[p]) != want.end()) pos.push_back(p);
        std::vector<int> perm;
        for (int lab : want) {
          for (size_t q = 0; q < pos.size(); ++q)
            if (h[pos[q]] == lab) { perm.push_back(int(q)); break; }
        }
        sign *= perm_parity(perm);
        for (size_t q = 0; q < pos.size(); ++q) h[pos[q]] = want[q];
      }
    }
  // rename dummies by first appearance
  std::map<int, int> rename;
  Canon c;
  c.sign = sign;
  for (auto &f : fs) {
    c.code.push_back(f.kind);
    c.code.push_back((int)f.groups.size());
    for (auto &g : f.groups) {
      c.code.push_back((int)g.size());
      for (int lab : g) {
        if (is_external(lab)) {
          c.code.push_back(lab);
        } else {
          auto it = rename.find(lab);
          if (it == rename.end()) it = rename.emplace(lab, make_label(64 + (int)rename.size(), lab_space(lab))).first;
          c.code.push_back(it->second);
        }
      }
    }
  }
  return c;
}

Canon canonical(std::vector<Factor> fs) {
  std::stable_sort(fs.begin(), fs.end(), [](const Factor &a, const Factor &b) { return a.kind < b.kind; });
  // permutations among factors of equal kind
  std::vector<int> order(fs.size());
  std::iota(order.begin(), order.end(), 0);
  Canon best;
  bool have = false;
  // enumerate by permuting within runs of equal kind
  std::vector<std::pair<int, int>> runs;
  for (size_t i = 0; i < fs.size();) {
    size_t j = i;
    while (j < fs.size() && fs[j].kind == fs[i].kind) ++j;
    runs.push_back({int(i), int(j)});
    i = j;
  }
  std::function<void(size_t)> rec = [&](size_t r) {
    if (r == runs.size()) {
      std::vector<Factor> arr;
      for (int k : order) arr.push_back(fs[k]);
      Canon c = canonical_fixed(arr);
      if (!have || c.code < best.code) { best = c; have = true; }
      return;
    }
    int b = runs[r].first, e = runs[r].second;
    std::sort(order.begin() + b, order.begin() + e);
    do { rec(r + 1); } while (std::next_permutation(order.begin() + b, order.begin() + e));
  };
  rec(0);
  return best;
}

std::vector<Factor> decode(const std::vector<int> &code) {
  std::vector<Factor> fs;
  size_t p = 0;
  while (p < code.size()) {
    Factor f;
    f.kind = code[p++];
    int ng = code[p++];
    for (int g = 0; g < ng; ++g) {
      int n = code[p++];
      std::vector<int> grp(code.begin() + p, code.begin() + p + n);
      p += n;
      f.groups.push_back(grp);
    }
    fs.push_back(f);
  }
  return fs;
}

// ---- enumeration of contractions ------------------------------------------------

void expand_into(int nh, int np, const std::vector<StringDef> &xs, Frac weight,
                 std::map<std::vector<int>, Frac> &acc) {
  for (const StringDef &hs : hamiltonian_strings()) {
    std::vector<const StringDef *> owners = {&hs};
    for (auto &x : xs) owners.push_back(&x);
    std::vector<SeqOp> seq;
    for (int k = 0; k < nh; ++k) seq.push_back({-1, SP_O, true, make_label(k, SP_O)});
    for (int k = np - 1; k >= 0; --k) seq.push_back({-1, SP_V, false, make_label(nh + k, SP_V)});
    for (int oi = 0; oi < (int)owners.size(); ++oi)
      for (auto &op : owners[oi]->ops) seq.push_back({oi, op.space, op.dag, op.slot});
    // balance check per space
    int bal[2] = {0, 0};
    for (auto &s : seq) bal[s.space] += qp_annihilator(s) ? 1 : -1;
    if (bal[0] || bal[1]) continue;
    Frac pref = weight;
    for (auto *o : owners) pref = pref * o->pref;
    const int nseq = (int)seq.size();
    std::vector<int> partner(nseq, -1);
    std::vector<int> creators;
    for (int i = nseq - 1; i >= 0; --i)
      if (!qp_annihilator(seq[i])) creators.push_back(i);
    std::function<void(size_t)> rec = [&](size_t ci) {
      if (ci == creators.size()) {
        // every owner > 0 must be joined to owner 0
        std::vector<bool> joined(owners.size(), false);
        std::vector<int> order;
        for (int i = 0; i < nseq; ++i) {
          if (!qp_annihilator(seq[i])) continue;
          int c = partner[i];
          int oa = seq[i].owner, oc = seq[c].owner;
          if (oa == 0 && oc > 0) joined[oc] = true;
          if (oc == 0 && oa > 0) joined[oa] = true;
          order.push_back(i);
          order.push_back(c);
        }
        for (size_t k = 1; k < owners.size(); ++k)
          if (!joined[k]) return;
        int sgn = perm_parity(order);
        // labels
        std::vector<std::vector<int>> slotlab(owners.size());
        for (size_t oi = 0; oi < owners.size(); ++oi) slotlab[oi].assign(owners[oi]->ops.size() + 2, -1);
        int dummy = 0;
        for (int i = 0; i < nseq; ++i) {
          if (!qp_annihilator(seq[i])) continue;
          int c = partner[i];
          int lab;
          if (seq[i].owner < 0) {
            lab = seq[i].tag;
          } else {
            lab = make_label(64 + dummy++, seq[i].space);
            slotlab[seq[i].owner][seq[i].tag] = lab;
          }
          slotlab[seq[c].owner][seq[c].tag] = lab;
        }
        std::vector<Factor> fs;
        for (size_t oi = 0; oi < owners.size(); ++oi) {
          Factor f;
          f.kind = owners[oi]->kind;
          for (auto &g : owners[oi]->groups) {
            std::vector<int> grp;
            for (int s : g) grp.push_back(slotlab[oi][s]);
            f.groups.push_back(grp);
          }
          fs.push_back(f);
        }
        Canon cn = canonical(fs);
        auto &slot = acc[cn.code];
        slot = slot + pref * Frac(cn.sign * sgn);
        return;
      }
      int c = creators[ci];
      for (int a = c - 1; a >= 0; --a) {
        if (!qp_annihilator(seq[a]) || partner[a] >= 0) continue;
        if (seq[a].space != seq[c].space || seq[a].owner == seq[c].owner) continue;
        partner[a] = c;
        rec(ci + 1);
        partner[a] = -1;
      }
    };
    rec(0);
  }
}

// Collect orbits under permutations of output holes / particles.
Equation reduce_orbits(int nh, int np, const std::map<std::vector<int>, Frac> &acc) {
  Equation eq;
  eq.nh = nh;
  eq.np = np;
  std::vector<int> hp(nh), pp(np);
  std::iota(hp.begin(), hp.end(), 0);
  std::iota(pp.begin(), pp.end(), 0);
  std::vector<std::pair<std::vector<int>, int>> group;  // (external id map, sign)
  do {
    do {
      std::vector<int> m(nh + np);
      for (int k = 0; k < nh; ++k) m[k] = hp[k];
      for (int k = 0; k < np; ++k) m[nh + k] = nh + pp[k];
      group.push_back({m, perm_parity(hp) * perm_parity(pp)});
    } while (std::next_permutation(pp.begin(), pp.end()));
  } while (std::next_permutation(hp.begin(), hp.end()));
  std::set<std::vector<int>> done;
  for (auto &kv : acc) {
    if (kv.second.zero() || done.count(kv.first)) continue;
    std::vector<int> rep;
    std::vector<std::vector<int>> members;
    int stab = 0;
    bool inconsistent = false;
    for (auto &gm : group) {
      std::vector<Factor> fs = decode(kv.first);
      for (auto &f : fs)
        for (auto &g : f.groups)
          for (int &lab : g)
            if (is_external(lab)) lab = make_label(gm.first[lab >> 1], lab_space(lab));
      Canon c = canonical(fs);
      if (c.code == kv.first) {
        ++stab;
        if (c.sign != gm.second) inconsistent = true;
      }
      members.push_back(c.code);
      if (rep.empty() || c.code < rep) rep = c.code;
    }
    for (auto &m : members) done.insert(m);
    auto it = acc.find(rep);
    if (it == acc.end() || it->second.zero()) continue;
    if (inconsistent) throw std::runtime_error("planner: inconsistent orbit with nonzero coefficient");
    Term t;
    t.coef = it->second.value() / double(stab);
    t.factors = decode(rep);
    eq.terms.push_back(t);
  }
  return eq;
}

struct TMulti { std::vector<int> ranks; Frac w; };

std::vector<TMulti> cluster_products(int maxn) {
  std::vector<TMulti> out;
  for (int n = 0; n <= maxn; ++n)
    for (int n3 = 0; n3 <= n; ++n3) {
      int n2 = n - n3;
      TMulti m;
      for (int k = 0; k < n2; ++k) m.ranks.push_back(2);
      for (int k = 0; k < n3; ++k) m.ranks.push_back(3);
      m.w = Frac(1, factorial(n2) * factorial(n3));
      out.push_back(m);
    }
  return out;
}

const int kEomSpaces[kEomVariants][3][2] = {
    {{1, 0}, {2, 1}, {3, 2}},  // IP
    {{0, 1}, {1, 2}, {2, 3}},  // EA
    {{2, 0}, {3, 1}, {4, 2}},  // DIP
    {{0, 2}, {1, 3}, {2, 4}},  // DEA
    {{1, 1}, {2, 2}, {3, 3}},  // EE
};

}  // namespace

void eom_component(int variant, int comp, int *nh, int *np) {
  *nh = kEomSpaces[variant][comp][0];
  *np = kEomSpaces[variant][comp][1];
}

Equation cc_equation(int rank) {
  std::map<std::vector<int>, Frac> acc;
  for (auto &m : cluster_products(4)) {
    std::vector<StringDef> xs;
    for (int r : m.ranks) xs.push_back(excitation_string(r == 2 ? TK_T2 : TK_T3, r, r));
    expand_into(rank, rank, xs, m.w, acc);
  }
  return reduce_orbits(rank, rank, acc);
}

namespace {

// Every full term of <mu_out| (H~ e^{T2+T3} R_in)_c |0> before orbit reduction.
std::map<std::vector<int>, Frac> eom_terms(int variant, int out_comp, int in_comp) {
  int nh, np, rh, rp;
  eom_component(variant, out_comp, &nh, &np);
  eom_component(variant, in_comp, &rh, &rp);
  std::map<std::vector<int>, Frac> acc;
  for (auto &m : cluster_products(3)) {
    std::vector<StringDef> xs;
    for (int r : m.ranks) xs.push_back(excitation_string(r == 2 ? TK_T2 : TK_T3, r, r));
    xs.push_back(excitation_string(TK_R1 + in_comp, rh, rp));
    expand_into(nh, np, xs, m.w, acc);
  }
  return acc;
}

}  // namespace

Equation eom_equation(int variant, int out_comp, int in_comp) {
  int nh, np;
  eom_component(variant, out_comp, &nh, &np);
  return reduce_orbits(nh, np, eom_terms(variant, out_comp, in_comp));
}

// Left product lambda_out <- L_in as the transpose of sigma_in <- R_out. With
// packed vectors, lambda[nu] = sum_{mu sorted} L[mu] d sigma[mu] / d r[nu];
// in dense antisymmetric tensors sum_{mu sorted} = 1 / (nh! np!) sum_mu, and
// d / d r[nu] sums d / d R[nu'] over the signed permutations nu' of nu. So
// each full term of sigma_in <- R_out becomes, with L[mu] on the old
// projection indices and the slots of R as the new projection indices, a term
// of weight c / (nh! np!); its copies under all signed permutations of the new
// hole and particle indices make the list closed under them, and the
// antisymmetriser the caller applies to the output then yields every signed
// permutation once, as the derivative requires.
Equation eom_left_equation(int variant, int out_comp, int in_comp) {
  int nh, np, rh, rp;
  eom_component(variant, in_comp, &nh, &np);   // projection of the right block = shape of L
  eom_component(variant, out_comp, &rh, &rp);  // input of the right block = shape of lambda
  const std::map<std::vector<int>, Frac> right = eom_terms(variant, in_comp, out_comp);
  const int rkind = TK_R1 + out_comp, lkind = TK_R1 + in_comp;
  const Frac norm(1, factorial(nh) * factorial(np));
  std::vector<int> hp(rh), pp(rp);
  std::map<std::vector<int>, Frac> acc;
  for (auto &kv : right) {
    if (kv.second.zero()) continue;
    std::vector<Factor> fs = decode(kv.first);
    int ri = -1;
    for (int k = 0; k < (int)fs.size(); ++k)
      if (fs[k].kind == rkind) {
        if (ri >= 0) throw std::runtime_error("planner: two EOM vectors in one term");
        ri = k;
      }
    if (ri < 0 || fs[ri].groups.size() != 2 || (int)fs[ri].groups[0].size() != rh ||
        (int)fs[ri].groups[1].size() != rp)
      throw std::runtime_error("planner: malformed EOM vector factor");
    const Factor rf = fs[ri];
    fs.erase(fs.begin() + ri);
    // old projection indices become dummies joined to L; R's slots become the
    // new projection indices (holes 0..rh-1, particles rh..)
    std::map<int, int> base;
    for (int id = 0; id < nh + np; ++id) {
      const int sp = id < nh ? SP_O : SP_V;
      base[make_label(id, sp)] = make_label(64 + 160 + id, sp);
    }
    std::vector<int> rslot;  // R slot label (after the rename above) per new index
    for (int k = 0; k < rh; ++k) rslot.push_back(rf.groups[0][k]);
    for (int k = 0; k < rp; ++k) rslot.push_back(rf.groups[1][k]);
    for (int &lab : rslot)
      if (base.count(lab)) lab = base[lab];
    Factor lf;
    lf.kind = lkind;
    lf.groups.resize(2);
    for (int id = 0; id < nh; ++id) lf.groups[0].push_back(base[make_label(id, SP_O)]);
    for (int id = nh; id < nh + np; ++id) lf.groups[1].push_back(base[make_label(id, SP_V)]);
    for (auto &f : fs)
      for (auto &g : f.groups)
        for (int &lab : g)
          if (base.count(lab)) lab = base[lab];
    fs.push_back(lf);
    std::iota(hp.begin(), hp.end(), 0);
    do {
      std::iota(pp.begin(), pp.end(), 0);
      do {
        std::map<int, int> ext;  // R slot label -> new projection index under this permutation
        for (int k = 0; k < rh; ++k) ext[rslot[k]] = make_label(hp[k], SP_O);
        for (int k = 0; k < rp; ++k) ext[rslot[rh + k]] = make_label(rh + pp[k], SP_V);
        std::vector<Factor> t = fs;
        for (auto &f : t)
          for (auto &g : f.groups)
            for (int &lab : g) {
              auto it = ext.find(lab);
              if (it != ext.end()) lab = it->second;
            }
        Canon c = canonical(t);
        auto &slot = acc[c.code];
        slot = slot + kv.second * norm * Frac(c.sign * perm_parity(hp) * perm_parity(pp));
      } while (std::next_permutation(pp.begin(), pp.end()));
    } while (std::next_permutation(hp.begin(), hp.end()));
  }
  return reduce_orbits(rh, rp, acc);
}

std::string equation_to_string(const Equation &eq) {
  static const char *names[] = {"f", "v", "t2", "t3", "r1", "r2", "r3"};
  std::ostringstream os;
  os.precision(17);
  os << eq.nh << " " << eq.np << " " << eq.terms.size() << "\n";
  for (auto &t : eq.terms) {
    os << t.coef;
    for (auto &f : t.factors) {
      os << " " << names[f.kind] << "[";
      for (size_t g = 0; g < f.groups.size(); ++g) {
        if (g) os << "|";
        for (size_t k = 0; k < f.groups[g].size(); ++k) {
          int lab = f.groups[g][k];
          if (k) os << ",";
          if (is_external(lab))
            os << ((lab_space(lab) == SP_O) ? "I" : "A") << (lab >> 1);
          else
            os << ((lab_space(lab) == SP_O) ? "o" : "v") << (lab >> 1);
        }
      }
      os << "]";
    }
    os << "\n";
  }
  return os.str();
}

// ---------------------------------------------------------------------------
// Contraction planning
// ---------------------------------------------------------------------------
namespace {

struct Node {
  Operand op;
  std::vector<std::vector<int>> anti;    // antisymmetric label groups (size >= 2)
  std::vector<std::vector<int>> packed;  // groups stored as sorted tuples (intermediates only)
  bool variable = false;                 // contains an EOM vector R
};

std::vector<std::vector<int>> factor_anti_groups(const Factor &f) {
  std::vector<std::vector<int>> out;
  for (auto &g : f.groups) {
    for (int sp = 0; sp < 2; ++sp) {
      std::vector<int> s;
      for (int lab : g)
        if (lab_space(lab) == sp) s.push_back(lab);
      if (s.size() >= 2) out.push_back(s);
    }
  }
  return out;
}

bool contains(const std::vector<int> &v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

double binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  double r = 1;
  for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
  return r;
}

// Split `labels` into groups: packable subsets given antisymmetric groups.
std::vector<DimGroup> make_groups(const std::vector<int> &labels,
                                  const std::vector<std::vector<int>> &antiA,
                                  const std::vector<std::vector<int>> *antiB, bool allow_pack,
                                  double *mult) {
  std::vector<DimGroup> out;
  std::vector<bool> used(labels.size(), false);
  if (allow_pack) {
    for (auto &ga : antiA) {
      std::vector<std::vector<int>> cands;
      if (antiB) {
        for (auto &gb : *antiB) {
          std::vector<int> s;
          for (int lab : labels)
            if (contains(ga, lab) && contains(gb, lab)) s.push_back(lab);
          cands.push_back(s);
        }
      } else {
        std::vector<int> s;
        for (int lab : labels)
          if (contains(ga, lab)) s.push_back(lab);
        cands.push_back(s);
      }
      for (auto &s : cands) {
        std::vector<int> free;
        for (int lab : s) {
          size_t p = std::find(labels.begin(), labels.end(), lab) - labels.begin();
          if (!used[p]) free.push_back(lab);
        }
        if (free.size() >= 2) {
          DimGroup g;
          g.space = lab_space(free[0]);
          g.k = (int)free.size();
          g.packed = true;
          std::sort(free.begin(), free.end());  // canonical tuple-to-label order
          g.labels = free;
          for (int lab : free) used[std::find(labels.begin(), labels.end(), lab) - labels.begin()] = true;
          *mult *= double(factorial(g.k));
          out.push_back(g);
        }
      }
    }
  }
  for (size_t p = 0; p < labels.size(); ++p) {
    if (used[p]) continue;
    DimGroup g;
    g.space = lab_space(labels[p]);
    g.k = 1;
    g.packed = false;
    g.labels = {labels[p]};
    out.push_back(g);
  }
  return out;
}

// Free dimensions of an intermediate: groups already packed in the operand stay
// packed; with pack_all every antisymmetric free group is packed as well.
std::vector<DimGroup> free_groups(const std::vector<int> &labels, const std::vector<std::vector<int>> &anti,
                                  const std::vector<std::vector<int>> &packed, bool pack_all) {
  std::vector<std::vector<int>> use = pack_all ? anti : packed;
  double dummy = 1;
  std::vector<DimGroup> out = make_groups(labels, use, nullptr, true, &dummy);
  return out;
}

bool subset_of_some(const std::vector<int> &g, const std::vector<std::vector<int>> &groups) {
  for (auto &h : groups) {
    bool all = true;
    for (int x : g)
      if (!contains(h, x)) { all = false; break; }
    if (all) return true;
  }
  return false;
}

double groups_size(const std::vector<DimGroup> &gs, int o, int v) {
  double s = 1;
  for (auto &g : gs) {
    int n = g.space == SP_O ? o : v;
    s *= g.packed ? binom(n, g.k) : std::pow(double(n), g.k);
  }
  return s;
}

}  // namespace

TermPlan plan_term(const Term &t, int nh, int np, int o, int v, double amortize, double cache_cap) {
  (void)nh; (void)np;
  std::vector<Node> nodes;
  for (auto &f : t.factors) {
    Node n;
    n.variable = f.kind >= TK_R1 && f.kind <= TK_R3;
    n.op.kind = f.kind;
    for (auto &g : f.groups)
      for (int lab : g) n.op.labels.push_back(lab);
    n.anti = factor_anti_groups(f);
    nodes.push_back(n);
  }
  TermPlan best;
  double best_cost = -1;

  // recursive search over merge orders
  std::function<void(std::vector<Node>, TermPlan, double)> rec = [&](std::vector<Node> cur, TermPlan plan, double cost) {
    if (best_cost >= 0 && cost >= best_cost) return;
    if (cur.size() == 1 && !plan.steps.empty()) {
      best = plan;
      best_cost = cost;
      return;
    }
    if (cur.size() == 1) {
      // single-factor term: scatter-add of one tensor
      Step s;
      s.a = cur[0].op;
      s.b.kind = -1;
      double mult = 1;
      s.mg = make_groups(cur[0].op.labels, cur[0].anti, nullptr, true, &mult);
      s.to_output = true;
      s.alpha = t.coef * mult;
      plan.steps.push_back(s);
      best = plan;
      best_cost = cost;
      return;
    }
    for (size_t i = 0; i < cur.size(); ++i)
      for (size_t j = i + 1; j < cur.size(); ++j) {
        const Node &A = cur[i], &B = cur[j];
        std::vector<int> kl, fa, fb;
        for (int lab : A.op.labels) (contains(B.op.labels, lab) ? kl : fa).push_back(lab);
        for (int lab : B.op.labels)
          if (!contains(A.op.labels, lab)) fb.push_back(lab);
        if (kl.empty() && cur.size() > 2) continue;  // avoid outer products while others remain
        // a packed group of an operand is either contracted whole with an operand
        // antisymmetric in it, or stays whole among the free indices
        bool ok = true;
        const Node *pairs[2][2] = {{&A, &B}, {&B, &A}};
        for (auto &pr : pairs) {
          for (auto &g : pr[0]->packed) {
            int in = 0;
            for (int x : g) in += contains(kl, x) ? 1 : 0;
            if (in != 0 && in != (int)g.size()) ok = false;
            if (in == (int)g.size() && !subset_of_some(g, pr[1]->anti)) ok = false;
          }
        }
        if (!ok) continue;
        bool last = cur.size() == 2;
        for (int pack_all = 0; pack_all < (last ? 1 : 2); ++pack_all) {
          Step s;
          s.a = A.op;
          s.b = B.op;
          double mult = 1;
          s.kg = make_groups(kl, A.anti, &B.anti, true, &mult);
          if (last) {
            s.mg = make_groups(fa, A.anti, nullptr, true, &mult);
            s.ng = make_groups(fb, B.anti, nullptr, true, &mult);
          } else {
            s.mg = free_groups(fa, A.anti, A.packed, pack_all != 0);
            s.ng = free_groups(fb, B.anti, B.packed, pack_all != 0);
          }
          s.to_output = last;
          s.alpha = last ? t.coef * mult : mult;
          double m = groups_size(s.mg, o, v), k = groups_size(s.kg, o, v), n = groups_size(s.ng, o, v);
          double step_cost = 2.0 * m * n * k + (last ? 0.0 : m * n);
          const bool var = A.variable || B.variable;
          if (!var && !last && amortize > 0 && m * n <= cache_cap) {
            s.constant = true;
            step_cost /= amortize;
          }
          TermPlan np2 = plan;
          Node C;
          if (!last) {
            int id = (int)np2.inter_labels.size();
            s.out_inter = id;
            std::vector<int> labs;
            std::vector<DimGroup> dims;
            for (auto *gs : {&s.mg, &s.ng})
              for (auto &g : *gs) {
                labs.insert(labs.end(), g.labels.begin(), g.labels.end());
                dims.push_back(g);
                if (g.packed) C.packed.push_back(g.labels);
              }
            np2.inter_labels.push_back(labs);
            np2.inter_dims.push_back(dims);
            C.op.kind = TK_INTERMEDIATE;
            C.op.inter = id;
            C.op.labels = labs;
            C.variable = var || !s.constant;
            for (auto *src : {&A, &B})
              for (auto &g : src->anti) {
                std::vector<int> s2;
                for (int lab : g)
                  if (contains(labs, lab)) s2.push_back(lab);
                if (s2.size() >= 2) C.anti.push_back(s2);
              }
          }
          np2.steps.push_back(s);
          std::vector<Node> nxt;
          for (size_t q = 0; q < cur.size(); ++q)
            if (q != i && q != j) nxt.push_back(cur[q]);
          if (!last) nxt.push_back(C);
          if (last) {
            if (best_cost < 0 || cost + step_cost < best_cost) {
              best = np2;
              best_cost = cost + step_cost;
            }
          } else {
            rec(nxt, np2, cost + step_cost);
          }
        }
      }
  };
  rec(nodes, TermPlan(), 0.0);
  if (best.steps.empty()) throw std::runtime_error("planner: no contraction order found");
  return best;
}


namespace {

int amp_priority(int kind) {
  switch (kind) {
    case TK_R3: return 6;
    case TK_R2: return 5;
    case TK_R1: return 4;
    case TK_T3: return 3;
    case TK_T2: return 2;
    default: return -1;
  }
}

std::vector<int> group_key(const std::vector<DimGroup> &gs) {
  std::vector<int> k;
  for (auto &g : gs) {
    k.push_back(g.packed ? 1 : 0);
    k.push_back((int)g.labels.size());
    k.insert(k.end(), g.labels.begin(), g.labels.end());
  }
  return k;
}

std::vector<DimGroup> relabel(std::vector<DimGroup> gs, const std::map<int, int> &m) {
  for (auto &g : gs)
    for (int &l : g.labels) {
      auto it = m.find(l);
      if (it != m.end()) l = it->second;
    }
  for (auto &g : gs)
    if (g.packed) std::sort(g.labels.begin(), g.labels.end());
  std::sort(gs.begin(), gs.end(), [](const DimGroup &a, const DimGroup &b) { return a.labels < b.labels; });
  return gs;
}

struct FuseInfo {
  bool ok = false;
  bool q_is_b = true;
  Operand p, q;             // operands, q with role labels
  std::vector<DimGroup> pfree, kg, qfree;  // role labels, canonical order
  std::map<int, int> to_role, from_role;
  bool p_constant = false;
  double alpha = 0;
  std::vector<int> key;
};

FuseInfo fuse_info(const TermPlan &pl, double amortize) {
  FuseInfo fi;
  if (pl.steps.empty()) return fi;
  const Step &f = pl.steps.back();
  if (!f.to_output || f.b.kind < 0) return fi;
  int pa = amp_priority(f.a.kind), pb = amp_priority(f.b.kind);
  if (std::max(pa, pb) < 0) return fi;
  fi.q_is_b = pb >= pa;
  const Operand &q = fi.q_is_b ? f.b : f.a;
  fi.p = fi.q_is_b ? f.a : f.b;
  std::vector<int> klabs;
  for (auto &g : f.kg) klabs.insert(klabs.end(), g.labels.begin(), g.labels.end());
  for (size_t i = 0; i < q.labels.size(); ++i) {
    int l = q.labels[i];
    if (std::find(klabs.begin(), klabs.end(), l) != klabs.end()) {
      int r = make_label(200 + (int)i, lab_space(l));
      fi.to_role[l] = r;
      fi.from_role[r] = l;
    }
  }
  fi.q = q;
  for (int &l : fi.q.labels) {
    auto it = fi.to_role.find(l);
    if (it != fi.to_role.end()) l = it->second;
  }
  fi.kg = relabel(f.kg, fi.to_role);
  fi.pfree = relabel(fi.q_is_b ? f.mg : f.ng, fi.to_role);
  fi.qfree = relabel(fi.q_is_b ? f.ng : f.mg, fi.to_role);
  if (fi.p.kind == TK_INTERMEDIATE) {
    fi.p_constant = false;
    for (auto &s : pl.steps)
      if (!s.to_output && s.out_inter == fi.p.inter) fi.p_constant = s.constant;
  } else {
    fi.p_constant = amortize > 0 && amp_priority(fi.p.kind) < 4;
  }
  fi.alpha = f.alpha;
  fi.key.push_back(q.kind);
  fi.key.push_back(fi.p_constant ? 1 : 0);
  fi.key.insert(fi.key.end(), fi.q.labels.begin(), fi.q.labels.end());
  fi.key.push_back(-1);
  for (auto *gs : {&fi.kg, &fi.pfree, &fi.qfree}) {
    auto k = group_key(*gs);
    fi.key.insert(fi.key.end(), k.begin(), k.end());
    fi.key.push_back(-2);
  }
  fi.ok = true;
  return fi;
}

}  // namespace

std::vector<TermPlan> fuse_plans(const std::vector<TermPlan> &plans, double amortize) {
  std::vector<FuseInfo> info;
  for (auto &p : plans) info.push_back(fuse_info(p, amortize));
  std::vector<TermPlan> out;
  std::vector<bool> used(plans.size(), false);
  for (size_t i = 0; i < plans.size(); ++i) {
    if (used[i]) continue;
    std::vector<size_t> members = {i};
    if (info[i].ok)
      for (size_t j = i + 1; j < plans.size(); ++j)
        if (!used[j] && info[j].ok && info[j].key == info[i].key) members.push_back(j);
    if (members.size() < 2) {
      out.push_back(plans[i]);
      used[i] = true;
      continue;
    }
    const FuseInfo &fi0 = info[i];
    TermPlan fused;
    std::vector<DimGroup> fdims = fi0.pfree;
    fdims.insert(fdims.end(), fi0.kg.begin(), fi0.kg.end());
    std::vector<int> flabs;
    for (auto &g : fdims) flabs.insert(flabs.end(), g.labels.begin(), g.labels.end());
    fused.inter_dims.push_back(fdims);
    fused.inter_labels.push_back(flabs);
    for (size_t m : members) {
      used[m] = true;
      const TermPlan &pl = plans[m];
      const FuseInfo &fi = info[m];
      const int base = (int)fused.inter_dims.size();
      fused.inter_dims.insert(fused.inter_dims.end(), pl.inter_dims.begin(), pl.inter_dims.end());
      fused.inter_labels.insert(fused.inter_labels.end(), pl.inter_labels.begin(), pl.inter_labels.end());
      auto shift = [&](Operand o) {
        if (o.kind == TK_INTERMEDIATE) o.inter += base;
        return o;
      };
      for (size_t k = 0; k + 1 < pl.steps.size(); ++k) {
        Step s = pl.steps[k];
        s.a = shift(s.a);
        s.b = shift(s.b);
        if (!s.to_output) s.out_inter += base;
        fused.steps.push_back(s);
      }
      Step ax;
      ax.a = shift(fi.p);
      ax.b.kind = -1;
      ax.to_output = false;
      ax.out_inter = 0;
      ax.alpha = fi.alpha;
      ax.constant = fi.p_constant;
      ax.mg = fdims;
      for (auto &g : ax.mg)
        for (int &l : g.labels) {
          auto it = fi.from_role.find(l);
          if (it != fi.from_role.end()) l = it->second;
        }
      fused.steps.push_back(ax);
    }
    Step fin;
    fin.a.kind = TK_INTERMEDIATE;
    fin.a.inter = 0;
    fin.a.labels = flabs;
    fin.b = fi0.q;
    fin.mg = fi0.pfree;
    fin.kg = fi0.kg;
    fin.ng = fi0.qfree;
    fin.to_output = true;
    fin.alpha = 1.0;
    fused.steps.push_back(fin);
    out.push_back(fused);
  }
  return out;
}

}  // namespace fnocc
