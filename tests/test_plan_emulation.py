"""Host test of the library's contraction plans (no GPU).

fnocc_plan_text dumps, for each term, the GEMM steps the CUDA engine runs:
operands, intermediates (with antisymmetric groups stored as sorted tuples),
row/contraction/column index groups (packed or not) and the coefficient with
its packing multiplicities. Here those steps are executed literally in numpy
— the gather-GEMM-scatter semantics of k_gather_gemm — and the antisymmetrised
result is compared with the oracle. Plans are built with the cost model at the
benchmark's sizes and executed on a small system (plans are size independent).
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import eom, fno, packing, wick

pkg = pytest.importorskip("paper_2509_14157_gb300")

TK = {0: "f", 1: "v", 2: "t2", 3: "t3", 4: "r1", 5: "r2", 6: "r3", 100: "X"}


def _groups(tok, i):
    n = int(tok[i])
    out = []
    for g in tok[i + 1:i + 1 + n]:
        sp, k, pk, labs = g.split(":")
        out.append((int(sp), int(k), pk == "1", [int(x) for x in labs.split(",")]))
    return out, i + 1 + n


def parse_plan(text):
    lines = text.strip().splitlines()
    nh, np_, nt = map(int, lines[0].split())
    terms, i = [], 1
    for _ in range(nt):
        _, nsteps, ninter = lines[i].split()
        i += 1
        inters = []
        for _ in range(int(ninter)):
            tok = lines[i].split()
            dims, _ = _groups(tok, 2)
            inters.append(dims)
            i += 1
        steps = []
        for _ in range(int(nsteps)):
            tok = lines[i].split()
            i += 1
            ak, ai, bk, bi, to_out, oi, const = map(int, tok[1:8])
            alpha = float(tok[8])
            j = tok.index("A") + 1
            alab = []
            while tok[j] != "B":
                alab.append(int(tok[j]))
                j += 1
            j += 1
            blab = []
            while tok[j] != "M":
                blab.append(int(tok[j]))
                j += 1
            mg, j = _groups(tok, j + 1)
            kg, j = _groups(tok, j + 1)
            ng, j = _groups(tok, j + 1)
            steps.append(dict(a=(ak, ai, alab), b=(bk, bi, blab), to_out=to_out, out=oi, alpha=alpha,
                              mg=mg, kg=kg, ng=ng, constant=const))
        terms.append((inters, steps))
    return nh, np_, terms


def _tuples(group, o, v):
    sp, k, packed, labs = group
    n = o if sp == 0 else v
    if packed:
        return [dict(zip(labs, t)) for t in itertools.combinations(range(n), k)]
    return [dict(zip(labs, t)) for t in itertools.product(range(n), repeat=k)]


def _assignments(groups, o, v):
    lists = [_tuples(g, o, v) for g in groups]
    out = []
    for combo in itertools.product(*lists) if lists else [()]:
        d = {}
        for c in combo:
            d.update(c)
        out.append(d)
    return out


class Emulator:
    def __init__(self, f, g, amps, o, v):
        self.f, self.g, self.amps, self.o, self.v = f, g, amps, o, v

    def read(self, kind, inter, labs, assign, inters):
        o = self.o
        if kind in (0, 1):
            idx = tuple(assign[l] + (0 if (l & 1) == 0 else o) for l in labs)
            return (self.f if kind == 0 else self.g)[idx]
        if kind == 100:
            arr, dims = inters[inter]
            idx = []
            for sp, k, packed, dl in dims:
                vals = tuple(assign[l] for l in dl)
                if packed:
                    n = o if sp == 0 else self.v
                    assert list(vals) == sorted(vals) and len(set(vals)) == k
                    idx.append(list(itertools.combinations(range(n), k)).index(vals))
                else:
                    idx.append(vals[0])
            return arr[tuple(idx)]
        return self.amps[TK[kind]][tuple(assign[l] for l in labs)]

    def run(self, plan):
        nh, np_, terms = plan
        o, v = self.o, self.v
        y = np.zeros((o,) * nh + (v,) * np_)
        for inter_dims, steps in terms:
            inters = {}
            for s in steps:
                ak, ai, alab = s["a"]
                rows = _assignments(s["mg"], o, v)
                if s["b"][0] < 0:
                    cmat = np.array([self.read(ak, ai, alab, r, inters) for r in rows])[:, None]
                    cols = [{}]
                else:
                    bk, bi, blab = s["b"]
                    ks = _assignments(s["kg"], o, v)
                    cols = _assignments(s["ng"], o, v)
                    amat = np.array([[self.read(ak, ai, alab, {**r, **k}, inters) for k in ks] for r in rows])
                    bmat = np.array([[self.read(bk, bi, blab, {**k, **c}, inters) for c in cols] for k in ks])
                    cmat = amat.reshape(len(rows), len(ks)) @ bmat.reshape(len(ks), len(cols))
                cmat = s["alpha"] * cmat
                if s["to_out"]:
                    for i, r in enumerate(rows):
                        for j, c in enumerate(cols):
                            a = {**r, **c}
                            y[tuple(a[(e << 1) | (0 if e < nh else 1)] for e in range(nh + np_))] += cmat[i, j]
                else:
                    # the producer writes the intermediate's dims positionally: mg groups, then ng groups
                    dims = inter_dims[s["out"]]
                    if s["out"] not in inters:
                        shape = [len(_tuples(d, o, v)) for d in dims]
                        inters[s["out"]] = (np.zeros(shape), dims)
                    arr = inters[s["out"]][0]
                    wgroups = s["mg"] + s["ng"]
                    assert len(wgroups) == len(dims)
                    for i, r in enumerate(rows):
                        for j, c in enumerate(cols):
                            a = {**r, **c}
                            idx = []
                            for d, wg in zip(dims, wgroups):
                                vals = tuple(a[l] for l in wg[3])
                                if d[2]:
                                    n = o if d[0] == 0 else v
                                    idx.append(list(itertools.combinations(range(n), d[1])).index(vals))
                                else:
                                    idx.append(vals[0])
                            arr[tuple(idx)] += cmat[i, j]
        out = np.zeros_like(y)
        for hp in itertools.permutations(range(nh)):
            for pp in itertools.permutations(range(np_)):
                sgn = np.linalg.det(np.eye(nh)[list(hp)]) if nh else 1.0
                sgn *= np.linalg.det(np.eye(np_)[list(pp)]) if np_ else 1.0
                out += round(sgn) * np.transpose(y, list(hp) + [nh + x for x in pp])
        return out


@pytest.fixture(scope="module")
def system():
    nocc, n = 2, 5  # o = 4, v = 6
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 17)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    t = {r: packing.unpack(synth.random_packed(packing.packed_size(r, r, o, v), 60 + r, 0.1), r, r, o, v)
         for r in (2, 3)}
    return ham, t


@pytest.mark.parametrize("rank", [1, 2, 3])
def test_cc_plans_execute_to_oracle(system, rank):
    ham, t = system
    o, v = ham["o"], ham["v"]
    amps = {"t1": np.zeros((o, v)), "t2": t[2], "t3": t[3]}
    emu = Emulator(ham["f"], ham["g"], amps, o, v)
    got = emu.run(parse_plan(pkg.plan_text(0, 0, rank, 0, o=10, v=30)))
    ref = wick.evaluate(wick.cc_terms(rank), rank, rank, ham["f"], ham["g"], amps, o, v)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_eom_plans_execute_to_oracle(system, variant):
    ham, t = system
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES[variant]
    rs = [packing.unpack(synth.random_packed(packing.packed_size(nh, np_, o, v), 70 + k, 0.3), nh, np_, o, v)
          for k, (nh, np_) in enumerate(comps)]
    amps = {"t1": np.zeros((o, v)), "t2": t[2], "t3": t[3], "r1": rs[0], "r2": rs[1], "r3": rs[2]}
    emu = Emulator(ham["f"], ham["g"], amps, o, v)
    ref = eom.sigma_dense(variant, ham["f"], ham["g"], o, v, amps["t1"], t[2], t[3], rs)
    for oc in range(3):
        got = sum(emu.run(parse_plan(pkg.plan_text(1, variant, oc, ic, o=10, v=50, amortize=100.0)))
                  for ic in range(3))
        assert np.max(np.abs(got - ref[oc])) < 1e-12, (variant, oc)


@pytest.fixture(scope="module")
def left_system():
    nocc, n = 2, 4  # o = v = 4: every component non-empty, quick oracle left products
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 19)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    t = {r: packing.unpack(synth.random_packed(packing.packed_size(r, r, o, v), 80 + r, 0.1), r, r, o, v)
         for r in (2, 3)}
    return ham, t


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_left_eom_plans_execute_to_oracle(left_system, variant):
    """Plans of the transposed (left) product blocks, executed step by step,
    against the oracle's L times the product matrix in the target sector."""
    ham, t = left_system
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES[variant]
    mask = eom.ms_mask(variant, o, v)
    lvec = synth.random_packed(len(mask), 37, 0.3) * mask
    ls = eom.split(variant, o, v, lvec)
    amps = {"t1": np.zeros((o, v)), "t2": t[2], "t3": t[3], "r1": ls[0], "r2": ls[1], "r3": ls[2]}
    emu = Emulator(ham["f"], ham["g"], amps, o, v)
    ref = eom.left_sigma_packed(variant, ham["f"], ham["g"], o, v, amps["t1"], t[2], t[3], lvec)
    got = []
    for oc, (nh, np_) in enumerate(comps):
        dense = sum(emu.run(parse_plan(pkg.plan_text(2, variant, oc, ic, o=10, v=50, amortize=100.0)))
                    for ic in range(3))
        got.append(packing.pack(dense, nh, np_, o, v))
    got = np.concatenate(got)
    assert np.max(np.abs(got[mask] - ref[mask])) < 1e-12 * max(1.0, np.max(np.abs(ref)))
