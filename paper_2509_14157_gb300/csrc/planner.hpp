// Symbolic planner: derives the projected equations of the method by Wick's
// theorem and turns every distinct term into GEMM-shaped contraction steps.
//
// Equations (arXiv 2509.14157):
//   CCSDT residual  <Phi^n| (H~ e^{T2+T3})_c |Phi_0>, n = 1..3   (Eq. 6)
//   EOM product     <mu| (H~ e^{T2+T3} R)_c |Phi_0>             (Eq. 1-4)
// with H~ = e^{-T1} H e^{T1} the T1-similarity-transformed Hamiltonian in
// normal order (general one-body f~ and antisymmetric two-body v~ with every
// occupied/virtual block), so T1 never appears explicitly.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace fnocc {

enum Space : int { SP_O = 0, SP_V = 1 };

// Tensor kinds that appear in terms.
enum TensorKind : int { TK_F = 0, TK_V = 1, TK_T2 = 2, TK_T3 = 3, TK_R1 = 4, TK_R2 = 5, TK_R3 = 6,
                        TK_INTERMEDIATE = 100 };

struct Frac {
  long long n = 0, d = 1;
  Frac() {}
  Frac(long long a, long long b = 1);
  Frac operator+(const Frac &o) const;
  Frac operator*(const Frac &o) const;
  bool zero() const { return n == 0; }
  double value() const { return double(n) / double(d); }
};

// A label is (id << 1) | space. Externals have ids 0..nh+np-1 (holes first).
inline int lab_space(int lab) { return lab & 1; }
inline int make_label(int id, int sp) { return (id << 1) | sp; }

struct Factor {
  int kind;                              // TensorKind
  std::vector<std::vector<int>> groups;  // antisymmetric slot groups, labels in slot order
};

struct Term {
  double coef;                 // numeric coefficient applied to the representative
  std::vector<Factor> factors;
};

// Term list of one projection: output holes nh, particles np.
struct Equation {
  int nh = 0, np = 0;
  std::vector<Term> terms;     // orbit representatives, coefficient already divided by |Stab|
};

// CCSDT: rank 1..3 residual (0 = energy) with T2, T3 clusters.
Equation cc_equation(int rank);
// EOM: variant 0..3 (IP, EA, DIP, DEA), output component and input component (0..2).
Equation eom_equation(int variant, int out_comp, int in_comp);
// Left EOM product block lambda_{out_comp} <- L_{in_comp}: the transpose of
// the right block sigma_{in_comp} <- R_{out_comp}; L enters as the EOM vector
// of component in_comp (the same tensor kinds as R).
Equation eom_left_equation(int variant, int out_comp, int in_comp);
// (nh, np) of component c of a variant.
// EOM variants: 0 IP, 1 EA, 2 DIP, 3 DEA, 4 EE (excitation energies)
constexpr int kEomVariants = 5;
void eom_component(int variant, int comp, int *nh, int *np);

std::string equation_to_string(const Equation &eq);

// ---------------------------------------------------------------------------
// Contraction plans
// ---------------------------------------------------------------------------

// One index group of a GEMM dimension: the slots (positions in the operand
// storage) it addresses, all of one space; packed = strictly increasing tuples.
struct DimGroup {
  int space;
  int k;                    // number of indices in the group
  bool packed;
  std::vector<int> labels;  // labels in tuple order
};

// Operand of a step: an input tensor or an intermediate.
struct Operand {
  int kind;                 // TensorKind or TK_INTERMEDIATE
  int inter = -1;           // intermediate id
  std::vector<int> labels;  // storage slot order
};

struct Step {
  Operand a, b;             // b.kind < 0 for a one-operand (copy) step
  bool constant = false;    // result independent of R (computed once per H-bar, cached)
  std::vector<DimGroup> mg, kg, ng;  // GEMM dims: rows from a, contraction, columns from b
  bool to_output = false;   // write into the output accumulator
  int out_inter = -1;       // else the intermediate it creates (dims: mg then ng; packed groups
                            // stored as sorted tuples and only ever consumed whole)
  double alpha = 1.0;       // coefficient incl. packing multiplicities
};

struct TermPlan {
  std::vector<Step> steps;
  std::vector<std::vector<int>> inter_labels;     // per intermediate: its labels in storage order
  std::vector<std::vector<DimGroup>> inter_dims;  // per intermediate: storage dims (packed groups kept whole)
};

// Builds the contraction steps of a term for output holes nh, particles np,
// sized with o and v (used by the cost model that orders contractions).
// amortize: steps whose operands do not contain an EOM vector R are computed
// once and cached, so the cost model charges them 1/amortize of their flops
// (0 = no caching, every step charged in full). Cached intermediates larger
// than cache_cap doubles are not cached.
TermPlan plan_term(const Term &t, int nh, int np, int o, int v, double amortize = 0.0,
                   double cache_cap = 0.0);

// Fuses terms whose last GEMM contracts the same amplitude operand Q (T2, T3
// or an EOM component R) in the same way: their other operands P_t are summed
// into one intermediate F = sum_t alpha_t P_t (the H-bar element) and one GEMM
// F x Q replaces the per-term GEMMs. amortize > 0 marks F as cached when every
// P_t is R-independent.
std::vector<TermPlan> fuse_plans(const std::vector<TermPlan> &plans, double amortize);

}  // namespace fnocc
