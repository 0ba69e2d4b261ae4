"""Oracle: Fock-space (determinant) definition of CC and EOM quantities, and
full configuration interaction.

This module takes the definitions literally, with no algebra: states are
vectors over all 2^M occupation-number strings of M spin orbitals, creation
and annihilation operators act on them with the usual Jordan-Wigner signs,
and

  * the CC residual of Eq. 6 is <mu| e^{-T} H e^{T} |Phi_0>,
  * the CC energy of Eq. 7 is <Phi_0| e^{-T} H e^{T} |Phi_0>,
  * the connected EOM product of Eq. 1-4 is
        sigma_mu = <mu| e^{-T} (H R - R H) e^{T} |Phi_0>
    which equals <mu|(H-bar R)_c|Phi_0> for any T because R contains only
    quasi-particle creators and commutes with T,

with e^{+-T} summed as a terminating Taylor series (T is nilpotent). FCI is
the dense diagonalisation of H in one (N, M_s) sector.

Sizes: M <= 14 spin orbitals (2^14 = 16384 states).

Parity: this is the definition itself; it is additionally pinned by the
closed forms in tests/test_oracle_pins.py (one-electron systems, Koopmans
limits).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


class FockSpace:
    def __init__(self, m):
        if m > 16:
            raise ValueError("Fock space limited to 16 spin orbitals")
        self.m = m
        self.dim = 1 << m
        self.states = np.arange(self.dim, dtype=np.int64)

    def string(self, ops, coef=1.0):
        """Sparse matrix of coef * (product of ops), ops listed left to right
        as (orbital, is_creator)."""
        cur = self.states.copy()
        sign = np.ones(self.dim)
        valid = np.ones(self.dim, dtype=bool)
        for p, dag in reversed(ops):
            bit = (cur >> p) & 1
            valid &= (bit == 0) if dag else (bit == 1)
            below = np.bitwise_count(cur & ((1 << p) - 1)).astype(np.int64)
            sign *= 1.0 - 2.0 * (below & 1)
            cur = cur ^ (1 << p)
        return sp.coo_matrix((coef * sign[valid], (cur[valid], self.states[valid])),
                             shape=(self.dim, self.dim))

    def assemble(self, terms):
        """Sum of strings: terms is an iterable of (coef, ops)."""
        rows, cols, vals = [], [], []
        for coef, ops in terms:
            if coef == 0.0:
                continue
            m = self.string(ops, coef)
            rows.append(m.row)
            cols.append(m.col)
            vals.append(m.data)
        if not rows:
            return sp.csr_matrix((self.dim, self.dim))
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.dim, self.dim)).tocsr()

    def hamiltonian(self, hso, gso):
        """Bare H = sum h_pq p^+ q + 1/4 sum <pq||rs> p^+ q^+ s r."""
        m = self.m
        terms = [(hso[p, q], [(p, True), (q, False)]) for p in range(m) for q in range(m)]
        for p, q in itertools.combinations(range(m), 2):
            for r, s in itertools.combinations(range(m), 2):
                terms.append((gso[p, q, r, s], [(p, True), (q, True), (s, False), (r, False)]))
        return self.assemble(terms)

    def operator(self, dense, hole_orbs, part_orbs, nh, np_):
        """sum over i1<..<i_nh, a1<..<a_np of dense[i.., a..] a1^+..a_np^+ i_nh..i1,
        where index k of the hole slots maps to orbital hole_orbs[k]."""
        terms = []
        for hs in itertools.combinations(range(len(hole_orbs)), nh):
            for ps in itertools.combinations(range(len(part_orbs)), np_):
                c = dense[hs + ps]
                if c == 0.0:
                    continue
                ops = [(part_orbs[a], True) for a in ps] + [(hole_orbs[i], False) for i in reversed(hs)]
                terms.append((c, ops))
        return self.assemble(terms)

    def vacuum(self, nocc_orbs):
        """Occupation-number vector of the reference |Phi_0> (the orbitals nocc_orbs filled)."""
        v = np.zeros(self.dim)
        v[sum(1 << p for p in nocc_orbs)] = 1.0
        return v

    def basis_coeff(self, vec, hole_orbs, part_orbs, ref_orbs):
        """Coefficient <mu|vec> for |mu> = a1^+..a_np^+ i_nh..i1 |Phi_0>."""
        ref = sum(1 << p for p in ref_orbs)
        ops = [(a, True) for a in part_orbs] + [(i, False) for i in reversed(hole_orbs)]
        cur = ref
        sign = 1.0
        for p, dag in reversed(ops):
            bit = (cur >> p) & 1
            if (dag and bit) or ((not dag) and not bit):
                return 0.0
            if bin(cur & ((1 << p) - 1)).count("1") & 1:
                sign = -sign
            cur ^= 1 << p
        return sign * vec[cur]


def _exp_apply(op, vec, sign=1.0, max_terms=64):
    out = vec.copy()
    term = vec.copy()
    for k in range(1, max_terms):
        term = sign * (op @ term) / k
        if not np.any(term):
            return out
        out += term
    raise RuntimeError("Taylor series of a nilpotent operator did not terminate")


class DefinitionOracle:
    """Residuals, energies and EOM products from their definitions for a
    spin-orbital Hamiltonian (bare hso, gso) whose first o orbitals are the
    occupied ones of the reference determinant."""

    def __init__(self, hso, gso, o):
        self.m = hso.shape[0]
        self.o = o
        self.v = self.m - o
        self.fs = FockSpace(self.m)
        self.h = self.fs.hamiltonian(hso, gso)
        self.occ = list(range(o))
        self.vir = list(range(o, self.m))
        self.ref = self.fs.vacuum(self.occ)

    def cluster(self, amps):
        """T = T1 + T2 + T3 from dense amplitude tensors (dict rank -> array)."""
        tot = None
        for r, dense in amps.items():
            op = self.fs.operator(dense, self.occ, self.vir, r, r)
            tot = op if tot is None else tot + op
        return tot

    def cc_residual(self, amps, rank):
        """Dense <Phi^rank| e^{-T} H e^{T} |Phi_0> as [holes..., particles...]."""
        t = self.cluster(amps)
        chi = _exp_apply(t, self.h @ _exp_apply(t, self.ref), -1.0)
        return self._project(chi, rank, rank)

    def cc_energy(self, amps, e_ref):
        """Correlation energy <Phi_0| e^{-T} H e^{T} |Phi_0> - E_ref (the definition behind Eq. 7)."""
        t = self.cluster(amps)
        chi = _exp_apply(t, self.h @ _exp_apply(t, self.ref), -1.0)
        return float(self.ref @ chi) - e_ref

    def eom_sigma(self, amps, r_ops, out_nh, out_np):
        """Connected <mu| e^{-T}(H R - R H) e^{T}|Phi_0> for R given as a list
        of (dense, nh, np) components."""
        t = self.cluster(amps)
        rop = None
        for dense, nh, np_ in r_ops:
            op = self.fs.operator(dense, self.occ, self.vir, nh, np_)
            rop = op if rop is None else rop + op
        psi = _exp_apply(t, self.ref)
        a = self.h @ (rop @ psi) - rop @ (self.h @ psi)
        chi = _exp_apply(t, a, -1.0)
        return self._project(chi, out_nh, out_np)

    def _project(self, vec, nh, np_):
        out = np.zeros((self.o,) * nh + (self.v,) * np_)
        for hs in itertools.product(range(self.o), repeat=nh):
            if len(set(hs)) < nh:
                continue
            for ps in itertools.product(range(self.v), repeat=np_):
                if len(set(ps)) < np_:
                    continue
                out[hs + ps] = self.fs.basis_coeff(vec, [self.occ[i] for i in hs],
                                                   [self.vir[a] for a in ps], self.occ)
        return out


def fci_energies(hso, gso, nelec, ms2, nroots=None):
    """Eigenvalues of the bare Hamiltonian in the sector with nelec electrons
    and 2*M_s = ms2 (spin orbitals alternate alpha/beta)."""
    m = hso.shape[0]
    fs = FockSpace(m)
    h = fs.hamiltonian(hso, gso)
    st = fs.states
    n_e = np.bitwise_count(st).astype(np.int64)  # signed: na - nb below may be negative
    alpha_mask = sum(1 << p for p in range(0, m, 2))
    na = np.bitwise_count(st & alpha_mask).astype(np.int64)
    nb = n_e - na
    sel = np.where((n_e == nelec) & (na - nb == ms2))[0]
    hs = h[sel][:, sel].toarray()
    ev = np.sort(np.linalg.eigvals(hs).real)
    return ev if nroots is None else ev[:nroots]
