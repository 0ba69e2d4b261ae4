"""Host-side tests of libfnocc that need no GPU.

  * the shared library loads and exports every function include/fnocc.h declares;
  * the equations the library's planner derives (T1-similarity-transformed
    CCSDT residuals and all twelve EOM product blocks) reproduce the oracle's
    Wick terms when evaluated on the CPU with T1 = 0;
  * xfno_extrapolate agrees with the oracle; calls fail with a status, not a
    crash, when no device is present.
"""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import synth
from oracle import eom, fno, packing, wick, xfno

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pkg = pytest.importorskip("paper_2509_14157_gb300")


def header_functions():
    text = open(os.path.join(ROOT, "include", "fnocc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[a-zA-Z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "sizeof")))


def test_library_exports_every_declared_symbol():
    lib = pkg.load_library()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each of them
    assert set(names) <= set(pkg.SIGNATURES)


def test_create_without_device_reports_status():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = pkg.load_library()
    h = ctypes.c_void_p()
    st = lib.fnocc_create(ctypes.byref(h), 0, None)
    assert st != 0 and not h.value


def _parse(text):
    lines = text.strip().splitlines()
    nh, np_, nt = map(int, lines[0].split())
    terms = []
    for ln in lines[1:1 + nt]:
        parts = ln.split()
        facs = []
        for p in parts[1:]:
            m = re.match(r"(\w+)\[(.*)\]", p)
            groups = [g.split(",") if g else [] for g in m.group(2).split("|")]
            facs.append((m.group(1), groups))
        terms.append((float(parts[0]), facs))
    return nh, np_, terms


def _perm_sign(p):
    p = list(p)
    s = 1
    for a in range(len(p)):
        while p[a] != a:
            b = p[a]
            p[a], p[b] = p[b], p[a]
            s = -s
    return s


def _evaluate(eq, f, g, amps, o, v):
    nh, np_, terms = eq
    letters = "abcdefghijklmnopqrstuvwxyzBCDEFGHJKLMNOPQRSTUVWXYZ"
    ext = ["I%d" % k for k in range(nh)] + ["A%d" % (nh + k) for k in range(np_)]
    y = np.zeros((o,) * nh + (v,) * np_)
    for coef, facs in terms:
        labs = {e: letters[i] for i, e in enumerate(ext)}
        subs, ops = [], []
        for name, groups in facs:
            flat = [l for gg in groups for l in gg]
            for l in flat:
                labs.setdefault(l, letters[len(labs)])
            subs.append("".join(labs[l] for l in flat))
            if name in ("f", "v"):
                sl = tuple(slice(0, o) if l[0] in "Io" else slice(o, None) for l in flat)
                ops.append((f if name == "f" else g)[sl])
            else:
                ops.append(amps[name])
        y += coef * np.einsum(",".join(subs) + "->" + "".join(labs[e] for e in ext), *ops, optimize=True)
    out = np.zeros_like(y)
    for hp in itertools.permutations(range(nh)):
        for pp in itertools.permutations(range(np_)):
            out += _perm_sign(hp) * _perm_sign(pp) * np.transpose(y, list(hp) + [nh + x for x in pp])
    return out


@pytest.fixture(scope="module")
def system():
    nocc, n = 2, 5
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 7)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    t = {r: packing.unpack(synth.random_packed(packing.packed_size(r, r, o, v), 3 + r, 0.1), r, r, o, v)
         for r in (2, 3)}
    return ham, t


@pytest.mark.parametrize("rank", [0, 1, 2, 3])
def test_planner_cc_equations_match_oracle(system, rank):
    ham, t = system
    o, v = ham["o"], ham["v"]
    amps = {"t1": np.zeros((o, v)), "t2": t[2], "t3": t[3]}
    got = _evaluate(_parse(pkg.equation_text(0, 0, rank)), ham["f"], ham["g"], amps, o, v)
    ref = wick.evaluate(wick.cc_terms(rank), rank, rank, ham["f"], ham["g"], amps, o, v)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_planner_eom_equations_match_oracle(system, variant):
    ham, t = system
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES[variant]
    rs = [packing.unpack(synth.random_packed(packing.packed_size(nh, np_, o, v), 11 + k, 0.3), nh, np_, o, v)
          for k, (nh, np_) in enumerate(comps)]
    amps = {"t1": np.zeros((o, v)), "t2": t[2], "t3": t[3], "r1": rs[0], "r2": rs[1], "r3": rs[2]}
    ref = eom.sigma_dense(variant, ham["f"], ham["g"], o, v, amps["t1"], t[2], t[3], rs)
    for oc in range(3):
        got = sum(_evaluate(_parse(pkg.equation_text(1, variant, oc, ic)), ham["f"], ham["g"], amps, o, v)
                  for ic in range(3))
        assert np.max(np.abs(got - ref[oc])) < 1e-12, (variant, oc)


@pytest.fixture(scope="module")
def left_system():
    # o = v = 4: every component of every variant is non-empty, and the
    # oracle's left product (one product per sector element) stays quick
    nocc, n = 2, 4
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 9)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    t = {r: packing.unpack(synth.random_packed(packing.packed_size(r, r, o, v), 13 + r, 0.1), r, r, o, v)
         for r in (2, 3)}
    return ham, t


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_planner_left_eom_equations_match_oracle(left_system, variant):
    """Left product blocks lambda_out <- L_in (the planner's transposed terms)
    against the oracle's L times the product matrix, in the target sector."""
    ham, t = left_system
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES[variant]
    mask = eom.ms_mask(variant, o, v)
    lvec = synth.random_packed(len(mask), 31, 0.3) * mask
    ls = eom.split(variant, o, v, lvec)
    amps = {"t1": np.zeros((o, v)), "t2": t[2], "t3": t[3], "r1": ls[0], "r2": ls[1], "r3": ls[2]}
    ref = eom.left_sigma_packed(variant, ham["f"], ham["g"], o, v, amps["t1"], t[2], t[3], lvec)
    got = []
    for oc, (nh, np_) in enumerate(comps):
        dense = sum(_evaluate(_parse(pkg.equation_text(2, variant, oc, ic)), ham["f"], ham["g"], amps, o, v)
                    for ic in range(3))
        got.append(packing.pack(dense, nh, np_, o, v))
    got = np.concatenate(got)
    # (the random T of this fixture does not conserve M_s, so only the sector is compared)
    assert np.max(np.abs(got[mask] - ref[mask])) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_plan_stats_are_consistent():
    """Host-only plan statistics: padded work covers the algorithmic work,
    the model time is at least the algorithmic work at the FP64 peak, and
    the DEA product's grouped flops match the algorithmic count the library
    reports for it (5.3e9 at o = 10, v = 30)."""
    peak = 152 * 2 * 2 * 2.07e9
    tot = padded = grouped = 0.0
    for oc in range(3):
        for ic in range(3):
            s = pkg.plan_stats(1, "dea", oc, ic, o=10, v=30)
            assert s["padded_flops"] >= s["grouped_flops"] >= 0
            assert s["model_seconds"] >= s["grouped_flops"] / peak * (1 - 1e-12)
            assert s["small_launch_flops"] <= s["grouped_flops"]
            tot += s["grouped_flops"] + s["other_flops"]
            padded += s["padded_flops"]
            grouped += s["grouped_flops"]
    assert 5.2e9 < tot < 5.45e9
    # the tile set keeps the padding of this product low (1.40 with 16-wide K tiles only)
    assert padded / grouped < 1.25
    with pytest.raises(ValueError):
        pkg.plan_stats(1, "dea", 3, 0)


def test_launch_descriptors_at_the_benchmark_size():
    """Every grouped step of every CCSDT rank and every right and left
    product block at the benchmark's size (o = 10, v = 30): the launch
    descriptors of all tile shapes (including the split reductions of the
    large steps) are consistent; the small steps' tables match the spin
    blocks element by element."""
    bad = sum(pkg.plan_selfcheck(0, 0, r, 0, 10, 30, 2e5) for r in range(1, 4))
    for kind in (1, 2):
        for var in ("ip", "ea", "dip", "dea", "ee"):
            for oc in range(3):
                for ic in range(3):
                    bad += pkg.plan_selfcheck(kind, var, oc, ic, 10, 30, 2e5)
    assert bad == 0


def test_plans_build_at_the_largest_workload():
    """Every CCSDT rank and every right and left product block builds its
    executable plan host-only at the largest workload (16 electrons, 41 kept
    virtuals: o = 16, v = 82), with 64-bit tables and grids in range, and
    its small grouped steps check out against the spin blocks."""
    o, v = 16, 82
    for rank in range(4):
        s = pkg.plan_stats(0, 0, rank, 0, o=o, v=v)
        assert s["padded_flops"] >= s["grouped_flops"] > 0 or rank == 0
    for kind in (1, 2):
        for var in ("ip", "ea", "dip", "ee"):
            for oc in range(3):
                for ic in range(3):
                    s = pkg.plan_stats(kind, var, oc, ic, o=o, v=v)
                    assert s["padded_flops"] >= s["grouped_flops"] >= 0
    assert pkg.plan_selfcheck(1, "ea", 2, 2, o, v, max_work=1e5) == 0


def test_xfno_matches_oracle():
    f = [0.999, 0.9975, 0.995]
    e = [-1.2001, -1.2004, -1.2011]
    assert abs(pkg.xfno_extrapolate(f, e) - xfno.extrapolate(f, e)) < 1e-14
    assert abs(pkg.xfno_extrapolate([1.0], [-3.0]) + 3.0) < 1e-15


@pytest.mark.parametrize("o,v", [(4, 6), (6, 4)])
def test_grouped_tasks_cover_the_spin_blocks_exactly(o, v):
    """Host-only plans of every CCSDT rank and every EOM block: the flat
    tables of the grouped tasks address exactly the operand offsets of the
    spin-allowed blocks, for every tile shape (no GPU)."""
    import paper_2509_14157_gb300 as pkg
    for rank in range(4):
        assert pkg.plan_selfcheck(0, 0, rank, 0, o, v) == 0, rank
    for kind in (1, 2):  # right and left (transposed) EOM products
        for var in ("ip", "ea", "dip", "dea", "ee"):
            for oc in range(3):
                for ic in range(3):
                    assert pkg.plan_selfcheck(kind, var, oc, ic, o, v) == 0, (kind, var, oc, ic)
