"""Oracle: term lists of coupled-cluster projections by Wick's theorem.

The paper prints no working equations (Eq. 1-7 only define the method), so
the oracle derives them mechanically: every projection it needs is a vacuum
expectation value

    < 0 | P  H  X_1 ... X_n | 0 >

of normal-ordered operator strings (P the de-excitation of the projection
determinant, H the normal-ordered Hamiltonian, X_k cluster operators T_m and,
for EOM, one R component). Wick's theorem gives it as the sum over all full
contractions; each contraction pairs a quasi-particle annihilator with a
quasi-particle creator further to the right in another string, and carries
the sign (-1)^(number of crossing pairs). Only connected terms are kept: H
must be joined to every X_k (the linked form of e^{-T} H e^{T} in Eq. 6-7 and
of (H-bar R)_c in Eq. 1-4).

Nothing here is factorised or reordered: each distinct term is one einsum
over dense antisymmetric tensors. Terms equal up to dummy relabelling and
antisymmetric slot exchange are merged.

Conventions (shared by the whole oracle)
  H = E_ref + sum f_pq {p^+ q} + 1/4 sum <pq||rs> {p^+ q^+ s r}
  T_m = (1/m!)^2 sum t[i1..im, a1..am] a1^+ .. am^+ im .. i1
  R with nh holes, np particles: 1/(nh! np!) sum r[h.., p..] p1^+..p_np^+ h_nh..h1
  |mu> = a1^+ .. a_np^+ i_nh .. i1 |0>,  <mu| = <0| i1^+ .. i_nh^+ a_np .. a1

Parity: pinned against the Fock-space definition oracle (oracle/detspace.py)
on random amplitudes and Hamiltonians, term sum by term sum.
"""
from __future__ import annotations

import functools
import itertools
import math
from collections import namedtuple
from fractions import Fraction

import numpy as np

Op = namedtuple("Op", "owner space dag label")


def _qp_ann(op):
    return (op.space == "o" and op.dag) or (op.space == "v" and not op.dag)


def _perm_sign(perm):
    perm = list(perm)
    s = 1
    for i in range(len(perm)):
        while perm[i] != i:
            j = perm[i]
            perm[i], perm[j] = perm[j], perm[i]
            s = -s
    return s


# --------------------------------------------------------------------------
# operator strings
# --------------------------------------------------------------------------

class Factor:
    """One normal-ordered operator string with its tensor."""

    def __init__(self, name, ops, groups, pref):
        self.name = name          # tensor name (e.g. 'f_ov', 'v_oovv', 't3', 'r2')
        self.ops = ops            # list of (space, dag, slot)
        self.groups = groups      # antisymmetric slot groups (tuples of slots)
        self.pref = pref          # Fraction prefactor


def fock_factor(ps, qs):
    """One-body part f_pq {p+ q} of the normal-ordered Hamiltonian, spaces ps, qs."""
    return Factor("f", [(ps, True, 0), (qs, False, 1)], ((0,), (1,)), Fraction(1))


def v_factor(sp):
    """Two-body part 1/4 <pq||rs> {p+ q+ s r}, spaces sp = "pqrs"."""
    p, q, r, s = sp
    return Factor("v", [(p, True, 0), (q, True, 1), (s, False, 3), (r, False, 2)],
                  ((0, 1), (2, 3)), Fraction(1, 4))


def amp_factor(name, nh, np_):
    """Excitation operator 1/(nh! np!) sum x a+.. i.. (T_n, or an EOM component)."""
    ops = [("v", True, nh + k) for k in range(np_)] + [("o", False, k) for k in reversed(range(nh))]
    groups = (tuple(range(nh)), tuple(range(nh, nh + np_)))
    return Factor(name, ops, groups, Fraction(1, math.factorial(nh) * math.factorial(np_)))


def hamiltonian_factors():
    """Every occupied/virtual block of the normal-ordered Hamiltonian."""
    out = [fock_factor(a, b) for a in "ov" for b in "ov"]
    out += [v_factor("".join(s)) for s in itertools.product("ov", repeat=4)]
    return out


def projector_ops(nh, np_):
    """Operators of <mu| with external labels I0.. (holes) and A0.. (particles)."""
    ops = [("o", True, "I%d" % k) for k in range(nh)]
    ops += [("v", False, "A%d" % k) for k in reversed(range(np_))]
    return ops


# --------------------------------------------------------------------------
# contraction enumeration
# --------------------------------------------------------------------------

def _full_contractions(seq):
    """All full pairings of the operator sequence. seq: list of Op."""
    ann = [i for i, op in enumerate(seq) if _qp_ann(op)]
    cre = [i for i, op in enumerate(seq) if not _qp_ann(op)]
    for sp in "ov":
        if sum(seq[i].space == sp for i in ann) != sum(seq[i].space == sp for i in cre):
            return
    used = [False] * len(seq)
    pairs = []

    def rec(k):
        if k == len(ann):
            yield list(pairs)
            return
        a = ann[k]
        for c in cre:
            if c > a and not used[c] and seq[c].space == seq[a].space and seq[c].owner != seq[a].owner:
                used[c] = True
                pairs.append((a, c))
                yield from rec(k + 1)
                pairs.pop()
                used[c] = False

    yield from rec(0)


def _crossing_sign(pairs):
    s = 1
    for x in range(len(pairs)):
        a1, c1 = pairs[x]
        for y in range(x + 1, len(pairs)):
            a2, c2 = pairs[y]
            if (a1 < a2 < c1 < c2) or (a2 < a1 < c2 < c1):
                s = -s
    return s


def _canon_fixed(tens, externals):
    occ = {}
    for ti, (_, groups) in enumerate(tens):
        for gi, g in enumerate(groups):
            for lab in g:
                occ.setdefault(lab, []).append((ti, gi))

    def partner(lab, ti, gi):
        if lab in externals:
            return (0, lab, 0)
        a, b = occ[lab]
        other = b if a == (ti, gi) else a
        return (1, other[0], other[1])

    sign = 1
    newg = [[list(g) for g in groups] for _, groups in tens]
    for ti in range(len(tens)):
        for gi in range(len(newg[ti])):
            g = newg[ti][gi]
            keys = [partner(l, ti, gi) for l in g]
            order = sorted(range(len(g)), key=lambda s: keys[s])
            sign *= _perm_sign(order)
            newg[ti][gi] = [g[s] for s in order]
    for ti in range(len(tens)):
        for gi in range(len(newg[ti])):
            g = newg[ti][gi]
            targets = []
            for lab in g:
                pk = partner(lab, ti, gi)
                if pk[0] == 1 and pk[1] > ti and (pk[1], pk[2]) not in targets:
                    targets.append((pk[1], pk[2]))
            for (tj, gj) in targets:
                want = [lab for lab in g if partner(lab, ti, gi)[1:] == (tj, gj)]
                h = newg[tj][gj]
                pos = [p for p, lab in enumerate(h) if lab in want]
                cur = [h[p] for p in pos]
                perm = [cur.index(l) for l in want]
                sign *= _perm_sign(perm)
                for p, lab in zip(pos, want):
                    h[p] = lab
    names = {}
    out = []
    for ti, (name, _) in enumerate(tens):
        gs = []
        for g in newg[ti]:
            gg = []
            for lab in g:
                if lab in externals:
                    gg.append(lab)
                else:
                    if lab not in names:
                        names[lab] = "%s%d" % (lab[0], len(names))
                    gg.append(names[lab])
            gs.append(tuple(gg))
        out.append((name, tuple(gs)))
    return tuple(out), sign


def canonical(tens, externals):
    """Canonical form of a product of antisymmetric tensors (up to dummy
    relabelling, slot exchange within groups and order of equal tensors)."""
    tens = sorted(tens, key=lambda t: t[0])
    blocks = [list(g) for _, g in itertools.groupby(range(len(tens)), key=lambda i: tens[i][0])]
    best = None
    for choice in itertools.product(*[itertools.permutations(b) for b in blocks]):
        order = [i for blk in choice for i in blk]
        key, sign = _canon_fixed([tens[i] for i in order], externals)
        if best is None or key < best[0]:
            best = (key, sign)
    return best


def expand(nh, np_, xs):
    """Connected terms of <mu(nh holes, np particles)| H X_1 .. X_n |0>.

    xs: list of Factor (cluster operators and at most one R). Returns a dict
    canonical-term -> Fraction coefficient (the exponential's 1/mult! for
    repeated T's must be folded in by the caller)."""
    externals = {"I%d" % k for k in range(nh)} | {"A%d" % k for k in range(np_)}
    acc = {}
    for hf in hamiltonian_factors():
        seq = [Op("P", sp, dg, lab) for sp, dg, lab in projector_ops(nh, np_)]
        slot_of = []
        owners = [hf] + list(xs)
        for oi, fac in enumerate(owners):
            for sp, dg, slot in fac.ops:
                seq.append(Op(oi, sp, dg, slot))
        pref = Fraction(1)
        for fac in owners:
            pref *= fac.pref
        for pairs in _full_contractions(seq):
            # connectivity: H (owner 0) joined to every other owner
            linked = set()
            for a, c in pairs:
                oa, oc = seq[a].owner, seq[c].owner
                if oa == 0 and oc != "P":
                    linked.add(oc)
                if oc == 0 and oa != "P":
                    linked.add(oa)
            if len(linked) != len(xs):
                continue
            labels = {}
            for k, (a, c) in enumerate(pairs):
                lab = seq[a].label if seq[a].owner == "P" else "%sd%d" % (seq[a].space, k)
                if seq[a].owner != "P":
                    labels[(seq[a].owner, seq[a].label)] = lab
                labels[(seq[c].owner, seq[c].label)] = lab
            tens = []
            for oi, fac in enumerate(owners):
                groups = tuple(tuple(labels[(oi, s)] for s in g) for g in fac.groups)
                tens.append((fac.name, groups))
            key, sign = canonical(tens, externals)
            acc[key] = acc.get(key, Fraction(0)) + pref * sign * _crossing_sign(pairs)
    return {k: c for k, c in acc.items() if c != 0}


# --------------------------------------------------------------------------
# equations of the method
# --------------------------------------------------------------------------

def _cluster_products(max_t, ranks=(1, 2, 3)):
    """Multisets of T ranks of size 0..max_t with their 1/prod(mult!) weight."""
    out = []
    for n in range(0, max_t + 1):
        for combo in itertools.combinations_with_replacement(ranks, n):
            w = Fraction(1)
            for r in set(combo):
                w /= math.factorial(combo.count(r))
            out.append((combo, w))
    return out


def _merge(dst, src, w):
    for k, c in src.items():
        dst[k] = dst.get(k, Fraction(0)) + w * c


@functools.lru_cache(maxsize=None)
def cc_terms(nh, t_ranks=(1, 2, 3)):
    """Terms of the CC projection <Phi^nh| (H e^T)_c |0> (Eq. 6; nh = 0 is the
    correlation energy of Eq. 7) for T = sum of the given ranks."""
    acc = {}
    for combo, w in _cluster_products(4, t_ranks):
        xs = [amp_factor("t%d" % r, r, r) for r in combo]
        _merge(acc, expand(nh, nh, xs), w)
    return tuple((k, c) for k, c in sorted(acc.items()) if c != 0)


# EOM operator spaces (reading of Eq. 3-4: three components per variant)
#   variant -> list of (holes, particles) of R1, R2, R3
# "ee" is the excitation-energy EOM-CCSDT (1h1p, 2h2p, 3h3p) that the
# paper's Sec. 1 builds the particle-number-changing variants on; the same
# product <mu| (H-bar R)_c |0> applies, R being an excitation operator.
EOM_SPACES = {
    "ip": [(1, 0), (2, 1), (3, 2)],
    "ea": [(0, 1), (1, 2), (2, 3)],
    "dip": [(2, 0), (3, 1), (4, 2)],
    "dea": [(0, 2), (1, 3), (2, 4)],
    "ee": [(1, 1), (2, 2), (3, 3)],
}


@functools.lru_cache(maxsize=None)
def eom_terms(variant, out_comp, in_comp, t_ranks=(1, 2, 3)):
    """Terms of sigma_out <- <mu_out| (H e^T R_in)_c |0> (Eq. 1-4)."""
    nh, np_ = EOM_SPACES[variant][out_comp]
    rh, rp = EOM_SPACES[variant][in_comp]
    acc = {}
    for combo, w in _cluster_products(3, t_ranks):
        xs = [amp_factor("t%d" % r, r, r) for r in combo] + [amp_factor("r%d" % (in_comp + 1), rh, rp)]
        _merge(acc, expand(nh, np_, xs), w)
    return tuple((k, c) for k, c in sorted(acc.items()) if c != 0)


# --------------------------------------------------------------------------
# evaluation
# --------------------------------------------------------------------------

_LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def _space(label):
    """Orbital space of a label: externals I*/A*, dummies o*/v*."""
    return "o" if label[0] in "Io" else "v"


def _operand(name, groups, f, g, amps, o):
    if name in ("f", "v"):
        sl = [slice(0, o) if _space(l) == "o" else slice(o, None) for gr in groups for l in gr]
        return f[tuple(sl)] if name == "f" else g[tuple(sl)]
    return amps[name]


def _subscripts(term, nh, np_):
    labs = {}
    out_labels = ["I%d" % k for k in range(nh)] + ["A%d" % k for k in range(np_)]
    for l in out_labels:
        labs[l] = _LETTERS[len(labs)]
    ins = []
    for _, groups in term:
        s = ""
        for gr in groups:
            for l in gr:
                if l not in labs:
                    labs[l] = _LETTERS[len(labs)]
                s += labs[l]
        ins.append(s)
    return ",".join(ins) + "->" + "".join(labs[l] for l in out_labels)


def evaluate(terms, nh, np_, f, g, amps, o, v):
    """Dense result tensor [holes..., particles...] of a term list."""
    out = np.zeros((o,) * nh + (v,) * np_)
    for term, coef in terms:
        ops = [_operand(name, groups, f, g, amps, o) for name, groups in term]
        if any(x.size == 0 for x in ops):
            continue
        out += float(coef) * np.einsum(_subscripts(term, nh, np_), *ops, optimize=True)
    return out


def evaluate_at(terms, nh, np_, f, g, amps, o, v, samples):
    """Result at selected output elements. samples: int array [S, nh+np]
    (hole indices 0..o-1 then particle indices 0..v-1)."""
    samples = np.asarray(samples, dtype=int).reshape(-1, nh + np_)
    out = np.zeros(len(samples))
    ext = ["I%d" % k for k in range(nh)] + ["A%d" % k for k in range(np_)]
    col = {l: k for k, l in enumerate(ext)}
    for term, coef in terms:
        labs = {"S": "Z"}
        ins, ops = [], []
        for name, groups in term:
            arr = _operand(name, groups, f, g, amps, o)
            flat = [l for gr in groups for l in gr]
            idx = []
            sub = "Z" if any(l in col for l in flat) else ""
            for ax, l in enumerate(flat):
                if l in col:
                    idx.append(samples[:, col[l]])
                else:
                    idx.append(slice(None))
                    if l not in labs:
                        labs[l] = _LETTERS[len(labs) - 1]
                    sub += labs[l]
            if sub.startswith("Z"):
                # gather external slots into a leading sample axis
                perm_axes = [ax for ax, l in enumerate(flat) if l in col] + \
                            [ax for ax, l in enumerate(flat) if l not in col]
                arr_t = np.transpose(arr, perm_axes)
                ext_idx = tuple(samples[:, col[flat[ax]]] for ax in perm_axes if flat[ax] in col)
                arr = arr_t[ext_idx]
            ins.append(sub)
            ops.append(arr)
        expr = ",".join(ins) + "->Z"
        if not any("Z" in s for s in ins):
            val = np.einsum(",".join(ins) + "->", *ops, optimize=True)
            out += float(coef) * val
        else:
            out += float(coef) * np.einsum(expr, *ops, optimize=True)
    return out
