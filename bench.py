"""Benchmark: seconds per converged EOM-CCSDT solve on one GB300 (FP64 path).

Workload (one step): the seeded synthetic closed-shell Hamiltonian with 10
electrons in 48 spatial orbitals (synth.hamiltonian(10, 48, seed)), frozen
natural orbitals kept at occupation >= 1e-4, the CCSDT ground state, and the
four lowest roots of IP-, EA-, DIP- and DEA-EOM-CCSDT (Davidson from the
Koopmans guess, residual 1e-8, |d omega| 1e-10). A step is 4 EOM solves; `value` is
step time / 4.

  value  device-resident inputs (h, eri already in HBM), device time of the
         steps from CUDA events on the library's stream.
  e2e    the same through the host-pointer C ABI call (host->device copy of
         h and eri from pinned host memory and the read-back of every result
         inside the timed region).
Between timed steps L2 is flushed by writing a 512 MB buffer.

  python bench.py [--steps K] [--warmup W] [--impl fnocc|reference]
  torchrun --nproc-per-node N bench.py --gpus N   (independent replicas)
"""
from __future__ import annotations

import argparse
import copy
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

NE, NORB, THRESHOLD, NROOTS = 10, 48, 1e-4, 4
VARIANTS = ("ip", "ea", "dip", "dea")
METRIC = "s per converged EOM-CCSDT solve"
# FP64 FMA issue derived from unit counts and clocks (2 FMA per clock per SM,
# 152 SMs, 2070 MHz max): reported beside the measured figure
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def measured_fp64_peak(device=0):
    """FP64 peak measured on this device by the library's probe
    (fnocc_fp64_peak): FMA chains and mma.sync m8n8k4, TFLOP/s."""
    import paper_2509_14157_gb300 as pkg
    fma, dmma = pkg.fp64_peak(device)
    return fma, dmma, "measured in this run (fnocc_fp64_peak: register-only FP64 FMA chains on every SM)"


def measured_bf16_peak():
    """Sustained dense BF16 tensor peak measured on this machine (TFLOP/s)."""
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"]), "measured (sustained cuBLAS bf16)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback (sustained bf16)"
# Iteration counts and algorithmic flops per evaluation of one converged step
# of this workload, as the library measured them on a GB300; the reference
# arm uses them to turn its timed oracle sample into seconds per solve.
REFERENCE_COUNTS = {"cc_iters": 21, "sigma": {"ip": 88, "ea": 89, "dip": 110, "dea": 74},
                    "flops_per_residual": 1.297e9,
                    "flops_per_sigma": {"ip": 1.94e8, "ea": 4.27e8, "dip": 4.77e8, "dea": 5.35e9}}


def config(threshold, seed):
    return {"workload": "FNO-EOM-CCSDT, %d electrons / %d orbitals synthetic closed-shell (seed %d), "
                        "FNO occupation >= %g, CCSDT + IP/EA/DIP/DEA x %d roots" % (NE, NORB, seed, threshold, NROOTS),
            "electrons": NE, "orbitals": NORB, "fno_threshold": threshold, "roots_per_variant": NROOTS,
            "variants": list(VARIANTS), "l2": "flushed between timed steps (512 MB write)",
            "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(s) > 4 + k and s[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _source_block(path, marker, back=0):
    """Lines of a C++ source from `back` lines above the line containing
    marker to the next closing brace at the marker's indentation."""
    lines = open(path).read().split("\n")
    at = next(i for i, l in enumerate(lines) if marker in l)
    indent = len(lines[at]) - len(lines[at].lstrip())
    end = next(i for i in range(at + 1, len(lines))
               if lines[i].startswith(" " * indent + "}") and len(lines[i]) - len(lines[i].lstrip()) == indent)
    return "\n".join(lines[at - back:end + 1])


def ggemm_source_sha():
    """sha256 of what the FP64 contraction kernel's DRAM traffic depends on:
    the k_ggemm template in gemm_grouped.cu (template line to closing brace)
    and the engine's offset-table builder in engine.cpp, which fixes the
    layout the kernel gathers from. The DRAM counters of a capture stay
    valid while both are unchanged."""
    csrc = os.path.join(HERE, "paper_2509_14157_gb300", "csrc")
    text = (_source_block(os.path.join(csrc, "gemm_grouped.cu"), "k_ggemm(const GTask", back=1) + "\n" +
            _source_block(os.path.join(csrc, "engine.cpp"), "long long add(DMap *map, const std::vector<DimGroup>"))
    return hashlib.sha256(text.encode()).hexdigest()


def read_traffic():
    """Per-launch DRAM bytes of the contraction kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(HERE, "profiles", "k_ggemm_fno_eom_c2.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"k_ggemm source sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram bytes per launch \(bench workload\):\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != ggemm_source_sha():
        return None
    return float(m_b.group(1))


# one term in SAMPLE_STRIDE of every block of the oracle's Wick term lists
# is timed (at least one per block), see OracleSample
SAMPLE_STRIDE = 16


class OracleSample:
    """The oracle, as it stands, on a bounded sample of one converged step.

    A converged step is the oracle's FNO setup, cc_iters CCSDT iterations
    (one residual evaluation of Eq. 6 each, plus the packing of the
    amplitudes) and, per variant, sigma_calls EOM products (Eq. 1-4, plus
    the unpacking of R and packing of sigma). Every residual and product is a
    sum over Wick terms evaluated as dense einsums, grouped in blocks (one
    per residual rank or product block); within a block the terms share the
    output shape. The sample: the FNO setup, the packing steps, and a seeded
    random choice of ceil(T / SAMPLE_STRIDE) of the T terms of every block
    (at least one), all timed on the host cores. A block is estimated as its
    output allocation plus (sampled time - allocation) x T / sampled terms;
    a residual or product as the sum of its blocks and packing steps. The
    GPU path's own call counts (iterations, products) turn these measured
    parts into seconds per converged solve."""

    def __init__(self, threshold, stride=SAMPLE_STRIDE, seed=0):
        import synth
        from oracle import fno as ofno, packing, wick
        self.packing, self.wick = packing, wick
        t0 = time.perf_counter()
        h, eri = synth.hamiltonian(NE, NORB, seed=0)
        act = ofno.fno_truncate(h, eri, NE // 2, threshold)
        self.t_fno = time.perf_counter() - t0
        self.f, self.g, self.o, self.v = act["f"], act["g"], act["o"], act["v"]
        o, v = self.o, self.v
        rng = np.random.default_rng(seed)
        self.amps = {"t%d" % r: packing.unpack(rng.normal(0, 0.01, math.comb(o, r) * math.comb(v, r)), r, r, o, v)
                     for r in (1, 2, 3)}
        self.blocks = {}  # (part, out_comp, in_comp) -> (terms, nh, np)
        for r in (1, 2, 3):
            self.blocks[("residual", r, 0)] = (wick.cc_terms(r), r, r)
        self.blocks[("residual", 0, 0)] = (wick.cc_terms(0), 0, 0)  # the energy of Eq. 7
        self.eom_amps = {}
        for var in VARIANTS:
            comps = wick.EOM_SPACES[var]
            for oc, (nh, np_) in enumerate(comps):
                for ic in range(3):
                    self.blocks[(var, oc, ic)] = (wick.eom_terms(var, oc, ic), nh, np_)
            self.eom_amps[var] = [rng.normal(0, 0.1, math.comb(o, nh) * math.comb(v, np_)) for nh, np_ in comps]
        # the work items: sampled terms of every block, then the packing steps
        self.items = []
        for key, (terms, nh, np_) in self.blocks.items():
            m = max(1, -(-len(terms) // stride))
            pick = np.sort(rng.choice(len(terms), size=m, replace=False))
            self.items.append(("terms", key, tuple(int(k) for k in pick)))
        self.items.append(("pack_t", None, None))
        for var in VARIANTS:
            self.items.append(("pack_r", var, None))
        self.times = {}

    def _amps_for(self, part):
        if part == "residual":
            return self.amps
        rs = [self.packing.unpack(x, nh, np_, self.o, self.v)
              for x, (nh, np_) in zip(self.eom_amps[part], self.wick.EOM_SPACES[part])]
        return dict(self.amps, r1=rs[0], r2=rs[1], r3=rs[2])

    def run(self, items):
        """Times the given work items on the host cores."""
        o, v, pk = self.o, self.v, self.packing
        cache = {}
        for kind, key, pick in items:
            if kind == "terms":
                terms, nh, np_ = self.blocks[key]
                if key[0] not in cache:
                    cache = {key[0]: self._amps_for(key[0])}  # dense inputs: setup, not timed
                amps = cache[key[0]]
                t0 = time.perf_counter()
                np.zeros((o,) * nh + (v,) * np_)
                t_alloc = time.perf_counter() - t0
                t0 = time.perf_counter()
                self.wick.evaluate(tuple(terms[k] for k in pick), nh, np_, self.f, self.g, amps, o, v)
                self.times[(kind, key)] = (t_alloc, time.perf_counter() - t0, len(pick), len(terms))
            elif kind == "pack_t":
                t0 = time.perf_counter()
                for r in (1, 2, 3):
                    pk.unpack(pk.pack(self.amps["t%d" % r], r, r, o, v), r, r, o, v)
                self.times[(kind, key)] = time.perf_counter() - t0
            else:
                comps = self.wick.EOM_SPACES[key]
                t0 = time.perf_counter()
                for x, (nh, np_) in zip(self.eom_amps[key], comps):
                    pk.pack(pk.unpack(x, nh, np_, o, v), nh, np_, o, v)
                self.times[(kind, key)] = time.perf_counter() - t0

    def seconds_sampled(self):
        tot = self.t_fno
        for k, x in self.times.items():
            tot += x[1] if k[0] == "terms" else x
        return tot

    def estimate(self, counts):
        """Oracle seconds per residual and per product (from the measured
        sample) and per converged solve (with the GPU path's call counts)."""
        part_s = {}
        for (kind, key), x in self.times.items():
            if kind == "terms":
                t_alloc, t, m, total = x
                part_s[key[0]] = part_s.get(key[0], 0.0) + t_alloc + max(t - t_alloc, 0.0) * total / m
            elif kind == "pack_t":
                part_s["residual"] = part_s.get("residual", 0.0) + x
            else:
                part_s[key] = part_s.get(key, 0.0) + x
        step = self.t_fno + counts["cc_iters"] * part_s["residual"] + sum(
            counts["sigma"][var] * part_s[var] for var in VARIANTS)
        return part_s, step / len(VARIANTS)


def cpu_baseline(threshold, gpu_counts):
    """The oracle timed on a bounded sample of the workload (OracleSample),
    scaled to seconds per converged solve with the GPU path's own iteration
    and product counts."""
    smp = OracleSample(threshold)
    smp.run(smp.items)
    part_s, per_solve = smp.estimate(gpu_counts)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": per_solve, "unit": "s", "cores": cores, "kind": "oracle",
            "sampled_seconds": round(smp.seconds_sampled(), 2),
            "oracle_s_per_ccsdt_iter": part_s["residual"],
            "oracle_s_per_sigma": {var: part_s[var] for var in VARIANTS},
            "sample": ("oracle (dense einsum over Wick terms, %d threads available) at o=%d, v=%d: FNO setup, "
                       "the packing steps, and 1 in %d Wick terms of every residual and product block (seeded, "
                       "at least one per block), %.1f s measured; each block scaled by its term count, each "
                       "residual / product by the GPU path's counts of this step (%d CCSDT iterations, "
                       "products %s); per converged solve = step / 4 (an estimate built from measured parts)"
                       % (cores, smp.o, smp.v, SAMPLE_STRIDE, smp.seconds_sampled(), gpu_counts["cc_iters"],
                          json.dumps(gpu_counts["sigma"])))}


def oracle_root_errors(roots, threshold, seed):
    """Total-energy error of every root against the roots the oracle wrote
    for this workload (tests/golden/c2_oracle.json, written by
    tests/golden/make_c2_golden.py), or None when no fixture covers it."""
    path = os.path.join(HERE, "tests", "golden", "c2_oracle.json")
    if seed != 0 or threshold != 1e-4 or (NE, NORB) != (10, 48) or not os.path.exists(path):
        return None
    gold = json.load(open(path))
    out = {"fixture": "tests/golden/c2_oracle.json", "per_root_err_eh": {}}
    for var in VARIANTS:
        if var not in gold.get("eom", {}) or var not in roots:
            continue
        ref = gold["e_ref"] + gold["e_ccsdt_corr"] + np.asarray(gold["eom"][var]["omega"])
        got = np.asarray(roots[var])[:len(ref)]
        out["per_root_err_eh"][var] = [float(x) for x in got - ref]
    errs = [abs(x) for v in out["per_root_err_eh"].values() for x in v]
    out["max_abs_err_eh"] = max(errs) if errs else None
    return out


def split_roofline(paths, step_s):
    """Tensor-core roofline of the split-product kernels of a profiled
    mixed-precision step: the tcgen05 BF16x3 kernel (k_ggemm_tc) and the
    mma.sync one (k_ggemm_bf16x3), each at six BF16 slice products per
    FP64-equivalent multiply-add, against the measured sustained BF16 peak."""
    peak, basis = measured_bf16_peak()
    out = {}
    for name in ("k_ggemm_tc", "k_ggemm_bf16x3"):
        ms_ = paths[name]["ms"] + paths[name + "_split+k_greduce"]["ms"]
        fl_ = paths[name]["flops"] + paths[name + "_split+k_greduce"]["flops"]
        n_ = paths[name]["launches"] + paths[name + "_split+k_greduce"]["launches"]
        ach = 6 * fl_ / (ms_ / 1e3) / 1e12 if ms_ > 0 else None
        out[name] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak if ach else None, "launches": n_, "ms": round(ms_, 3),
                     "share_of_step": (ms_ / 1e3) / step_s if step_s else None}
    out["peak_basis"] = basis + "; six BF16 slice products per FP64-equivalent multiply-add"
    out["paths"] = {k: {"ms": round(x["ms"], 3), "launches": x["launches"]} for k, x in paths.items()}
    return out


def replica_seed(rank):
    """Independent replicas: every rank solves its own seeded system (no
    collective on the data path)."""
    return rank


def max_over_ranks(seconds, world, device=None):
    """Whole-job time of replicas: the slowest rank's (all-reduce MAX)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """The reference arm: the oracle (the paper ships no code) on the host
    cores. Setup (oracle FNO, dense inputs, term derivation) is untimed; each
    warm-up step evaluates one sampled term; the timed steps share the
    OracleSample work items round-robin, so that the K steps together time
    the whole sample once. value = the oracle's seconds per converged solve
    estimated from those measured parts with the GPU path's call counts of
    this workload (REFERENCE_COUNTS); ms_per_step = the measured wall time
    of one timed step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    counts = REFERENCE_COUNTS
    t_all = time.time()
    smp = OracleSample(args.threshold)
    first = [it for it in smp.items if it[0] == "terms"][:1]
    for _ in range(args.warmup):
        smp.run(first)
    steps = max(1, args.steps)
    share = [smp.items[k::steps] for k in range(steps)]
    step_s = []
    for k in range(steps):
        t0 = time.perf_counter()
        smp.run(share[k])
        step_s.append(time.perf_counter() - t0)
    part_s, value = smp.estimate(counts)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    base = {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
            "sampled_seconds": round(smp.seconds_sampled(), 2),
            "oracle_s_per_ccsdt_iter": part_s["residual"],
            "oracle_s_per_sigma": {var: part_s[var] for var in VARIANTS},
            "sample": ("oracle at o=%d, v=%d: FNO setup, packing steps and 1 in %d Wick terms of every residual "
                       "and product block, timed over %d steps (%.1f s); scaled by term counts and by the GPU "
                       "path's counts of a converged step (%d CCSDT iterations, products %s); per converged "
                       "solve = step / 4 (an estimate built from measured parts)"
                       % (smp.o, smp.v, SAMPLE_STRIDE, steps, sum(step_s), counts["cc_iters"],
                          json.dumps(counts["sigma"])))}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_s) / steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config(args.threshold, 0), precision="fp64"),
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.time() - t_all}
    print(json.dumps(line), flush=True)


def run_solve_only(args):
    """One variant's converged solve at the workload's size: FNO, CCSDT, then
    the variant's NROOTS lowest roots (warm-up solve first, then the timed
    one); wall-clock seconds of the synchronous calls, products, iterations
    and algorithmic flops."""
    import paper_2509_14157_gb300 as pkg
    import synth
    ne, norb, thr, nroots = (PC_NE, PC_NORB, PC_THRESHOLD, PC_ROOTS) if args.large else (
        NE, NORB, args.threshold, NROOTS)
    h, eri = synth.hamiltonian(ne, norb, seed=0)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, ne // 2, thr)
    kw = (dict(precision="fp64") if args.precision == "fp64"
          else dict(precision=args.precision, switch_tol=0.0, tol_res=1e-6, tol_e=1e-8))
    t0 = time.perf_counter()
    cc = ctx.ccsdt_solve(precision="mixed" if args.large and args.precision != "fp64" else "fp64")
    t_cc = time.perf_counter() - t0
    kw["left"] = args.left
    if not args.large:  # warm solve (plans, cached pieces); the larger system times its first solve
        ctx.eom_solve(args.solve_only, nroots, **kw)
    f0 = ctx.flops
    t0 = time.perf_counter()
    r = ctx.eom_solve(args.solve_only, nroots, **kw)
    dt = time.perf_counter() - t0
    o, v, _ = ctx.dims()
    print(json.dumps({"solve_only": args.solve_only, "left": args.left, "precision": args.precision, "seconds": dt,
                      "system": {"electrons": ne, "orbitals": norb, "fno_threshold": thr, "o": o, "v": v,
                                 "roots": nroots, "dim": int(sum(ctx.eom_sizes(args.solve_only)))},
                      "ccsdt_seconds": t_cc, "energies": [float(x) for x in r["energies"]],
                      "sigma_calls": r["sigma_calls"], "iters": r["iters"], "converged": r["converged"],
                      "omegas": [float(x) for x in r["omegas"]], "ccsdt_iters": cc["iters"],
                      "tflops": (ctx.flops - f0) / dt / 1e12}), flush=True)
    ctx.close()


def run_sigma_only(args):
    """Profiling case: FNO setup, random amplitudes, two warm sigma products of
    one variant (the second with the R-independent intermediates cached, as
    inside a Davidson solve), then one more inside the NVTX range "sig"."""
    import torch
    import paper_2509_14157_gb300 as pkg
    import synth
    ne, norb, thr = ((PC_NE, PC_NORB, PC_THRESHOLD) if args.large else
                     (MID_NE, MID_NORB, MID_THRESHOLD) if args.mid else (NE, NORB, args.threshold))
    h, eri = synth.hamiltonian(ne, norb, seed=0)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, ne // 2, thr)
    rng = np.random.default_rng(0)
    ctx.set_amplitudes(*[rng.normal(0, 0.01, s) for s in ctx.amp_sizes()])
    ctx.set_precision(args.precision)
    if args.tile_shape >= 0:
        ctx.set_tile_shape(args.tile_shape)
    dim = sum(ctx.eom_sizes(args.sigma_only))
    product = ctx.eom_left_sigma_dev if args.left else ctx.eom_sigma_dev
    x = torch.from_numpy(rng.normal(0, 0.1, dim)).cuda()
    s = torch.empty_like(x)
    for _ in range(args.warm):
        product(args.sigma_only, x.data_ptr(), s.data_ptr())
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("sig")
    t0 = time.perf_counter()
    product(args.sigma_only, x.data_ptr(), s.data_ptr())
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"sigma_only": args.sigma_only, "left": args.left, "precision": args.precision, "seconds": dt,
                      "flops_all_calls": ctx.flops}), flush=True)
    ctx.close()


BATCH_ROOTS = 3


def batch_systems(count=16):
    """Uneven seeded systems: 8, 10 or 12 electrons, 8-14 kept natural
    virtuals (nkeep), 6 dropped virtuals beyond them. (With six electrons the
    IP sector holds only three principal states: a fourth root would be a
    satellite, which is not the workload here.)"""
    import synth
    out = []
    for s in range(count):
        ne = 8 + 2 * (s % 3)
        kept = 8 + (3 * s) % 7
        h, eri = synth.hamiltonian(ne, ne // 2 + kept + 6, seed=100 + s)
        out.append(dict(h=h, eri=eri, nocc=ne // 2, nkeep=kept))
    return out


def batch_systems_large(count=32):
    """Uneven seeded systems of the larger batch: 6-14 electrons, 20-40 kept
    natural virtuals (nkeep), 8 dropped virtuals beyond them."""
    import synth
    out = []
    for s in range(count):
        ne = 6 + 2 * (s % 5)
        kept = 20 + (13 * s) % 21
        h, eri = synth.hamiltonian(ne, ne // 2 + kept + 8, seed=200 + s)
        out.append(dict(h=h, eri=eri, nocc=ne // 2, nkeep=kept))
    return out


def run_batch(args):
    """Throughput over many independent systems: fnocc_batch_solve with 4
    workers (one context and stream each) against the same call with one
    worker. Every system's roots must agree. Default: 16 small systems, IP
    and EA x 3 roots, FP64. --batch-large: 32 systems of 6-14 electrons and
    20-40 kept virtuals, IP and EA x 4 roots, BF16x3 products with FP64
    refinement (CCSDT below 1e-6, Davidson below 1e-5)."""
    import paper_2509_14157_gb300 as pkg
    large = args.batch_large
    systems = batch_systems_large() if large else batch_systems()
    variants = ["ip", "ea"]
    nroots = 4 if large else BATCH_ROOTS
    prec = "mixed" if large else "fp64"
    pkg.batch_solve(systems[:2], variants, nroots, nworkers=2, precision=prec)  # warm: library, plans
    t0 = time.perf_counter()
    om1, info1 = pkg.batch_solve(systems, variants, nroots, nworkers=1, precision=prec)
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    om4, info4 = pkg.batch_solve(systems, variants, nroots, nworkers=4, precision=prec)
    t_bat = time.perf_counter() - t0
    ok = [i for i, (a, b) in enumerate(zip(info1, info4)) if a["status"] == 0 and b["status"] == 0]
    solves = len(ok) * len(variants)
    diff = float(np.max(np.abs(om1[ok] - om4[ok]))) if ok else None
    print(json.dumps({"metric": METRIC + " (batched independent systems)", "value": t_bat / max(solves, 1),
                      "unit": "s", "higher_is_better": False, "sequential_value": t_seq / max(solves, 1),
                      "speedup": t_seq / t_bat if t_bat > 0 else None, "systems": len(systems),
                      "converged_systems": len(ok), "statuses": [i["status"] for i in info4],
                      "messages": {str(s): i["message"] for s, i in enumerate(info4) if i["status"] != 0},
                      "workers": 4, "max_root_diff_eh": diff,
                      "config": ({"workload": "32 seeded systems, 6-14 electrons, 20-40 kept natural virtuals "
                                              "(nkeep), IP and EA x 4 roots",
                                  "precision": "BF16x3 products, FP64 refinement"} if large else
                                 {"workload": "16 seeded systems, 8/10/12 electrons, 8-14 kept natural virtuals "
                                              "(nkeep), IP and EA x 3 roots", "precision": "fp64"}),
                      "data": "synthetic"}), flush=True)


# larger system for the split-product accuracy check: 41 kept natural virtuals
PC_NE, PC_NORB, PC_THRESHOLD, PC_ROOTS, PC_VARIANTS = 16, 80, 1e-6, 6, ("ip", "ea", "dip")
# profiling case between the two (--sigma-only V --mid): 12 electrons / 60
# orbitals, FNO 1e-4 (17 kept natural virtuals, o = 12, v = 34); a DEA
# product holds a few GB on the device
MID_NE, MID_NORB, MID_THRESHOLD = 12, 60, 1e-4


def run_precision_check(args):
    """Accuracy and speed of the split-product kinds on the larger system
    (16 electrons / 80 orbitals, FNO occupation >= 1e-6: 41 kept natural
    virtuals, o = 16 and v = 82 spin orbitals), 6 roots of IP, EA and DIP.
    CCSDT in FP64, then in BF16x3 with FP64 refinement below 1e-6 (both from
    MP2 amplitudes); then every variant's Davidson solve in FP64 (residual
    1e-8) and kept in each split kind throughout (residual 1e-6, the 1e-6 Eh
    target), each from the same converged amplitudes. Reports per-root total
    energy errors of the split kinds against the FP64 solve and wall-clock
    seconds of the synchronous library calls; one JSON line per finished
    part, then a summary line. DEA (--pc-variants dea) fits at this size
    (dense R3 work tensor and accumulator 93 GB each, sector-compressed
    Davidson subspace) but its FP64 solve takes about a quarter of an hour,
    so it is run on request."""
    import paper_2509_14157_gb300 as pkg
    import synth

    def emit(d):
        print(json.dumps(d), flush=True)

    h, eri = synth.hamiltonian(PC_NE, PC_NORB, seed=0)
    ctx = pkg.Context(0)
    t0 = time.perf_counter()
    fi = ctx.fno_truncate(h, eri, PC_NE // 2, PC_THRESHOLD)
    o, v, _ = ctx.dims()
    summary = {"mode": "precision_check", "electrons": PC_NE, "orbitals": PC_NORB, "fno_threshold": PC_THRESHOLD,
               "nkept": fi["nkept"], "o": o, "v": v, "roots": PC_ROOTS, "fno_seconds": time.perf_counter() - t0,
               "data": "synthetic", "ccsdt": {}, "eom": {}}
    for prec in ("fp64", "mixed"):
        t0 = time.perf_counter()
        r = ctx.ccsdt_solve(precision=prec, switch_tol=1e-6)
        part = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "iters_mixed": r["iters_mixed"],
                "e_corr": r["e_corr"], "converged": r["converged"]}
        summary["ccsdt"][prec] = part
        emit({"part": "ccsdt", "precision": prec, **part})
    summary["ccsdt"]["e_corr_diff"] = summary["ccsdt"]["mixed"]["e_corr"] - summary["ccsdt"]["fp64"]["e_corr"]
    variants = tuple(args.pc_variants.split(",")) if args.pc_variants else PC_VARIANTS
    kinds = tuple(args.pc_kinds.split(",")) if args.pc_kinds else ("mixed", "mixed_tf32")
    for var in variants:
        res = {}
        for prec in ("fp64",) + kinds:
            kw = (dict(precision="fp64") if prec == "fp64"
                  else dict(precision=prec, switch_tol=0.0, tol_res=1e-6, tol_e=1e-8))
            t0 = time.perf_counter()
            r = ctx.eom_solve(var, PC_ROOTS, **kw)
            res[prec] = {"seconds": time.perf_counter() - t0, "sigma_calls": r["sigma_calls"],
                         "converged": r["converged"], "energies": [float(x) for x in r["energies"]]}
            emit({"part": "eom", "variant": var, "precision": prec, **res[prec]})
        ref = np.asarray(res["fp64"]["energies"])
        for prec in kinds:
            err = np.asarray(res[prec]["energies"]) - ref
            res[prec]["max_abs_err_eh"] = float(np.max(np.abs(err)))
            res[prec]["speedup_vs_fp64"] = res["fp64"]["seconds"] / res[prec]["seconds"]
        summary["eom"][var] = res
    emit(summary)
    ctx.close()


# XFNO check: the paper's three cumulative occupation thresholds (OCCT) and
# the untruncated space
XC_OCCT = (0.999, 0.9975, 0.995)


def run_xfno_check(args):
    """The FNO / XFNO pipeline end to end on the benchmarked system (10
    electrons / 48 orbitals): FNO with the paper's three cumulative
    occupation thresholds (OCCT 99.9 / 99.75 / 99.5 %, Sec. 2), and the
    untruncated space (threshold 0), each followed by CCSDT and 4 roots of
    IP, EA, DIP and DEA (BF16x3 products with FP64 refinement, so the
    roots carry the FP64 solution's accuracy). Reports per root the total
    energy of every truncation, its error against the untruncated energy
    (the paper's M2 - M1 at OCCT 99.9 %), the XFNO extrapolation of the
    three (least-squares line in the kept occupation fraction evaluated at
    1, xfno_extrapolate; the paper's M3) and its error, and the same for
    the ground state; one JSON line per finished part, then a summary."""
    import paper_2509_14157_gb300 as pkg
    import synth

    def emit(d):
        print(json.dumps(d), flush=True)

    h, eri = synth.hamiltonian(NE, NORB, seed=0)
    runs = [("occt", t) for t in XC_OCCT] + [("abs", 0.0)]
    res = {}
    for crit, thr in runs:
        ctx = pkg.Context(0)
        t0 = time.perf_counter()
        fi = ctx.fno_truncate(h, eri, NE // 2, thr, criterion=crit)
        cc = ctx.ccsdt_solve(precision="mixed", switch_tol=1e-6)
        o, v, e_ref = ctx.dims()
        part = {"criterion": crit, "threshold": thr, "nkept": fi["nkept"], "kept_fraction": fi["kept_fraction"],
                "o": o, "v": v, "e_ccsdt": cc["e_tot"], "ccsdt_converged": cc["converged"], "eom": {}}
        for var in VARIANTS:
            r = ctx.eom_solve(var, NROOTS, precision="mixed", switch_tol=1e-5)
            part["eom"][var] = {"energies": [float(x) for x in r["energies"]], "converged": r["converged"]}
        part["seconds"] = time.perf_counter() - t0
        res[(crit, thr)] = part
        emit({"part": "fno", **part})
        ctx.close()
    full = res[("abs", 0.0)]
    trunc = [res[("occt", t)] for t in XC_OCCT]
    f = [p["kept_fraction"] for p in trunc]
    summary = {"mode": "xfno_check", "electrons": NE, "orbitals": NORB, "data": "synthetic",
               "occt": list(XC_OCCT), "kept": [p["nkept"] for p in trunc], "kept_fraction": f,
               "untruncated_nkept": full["nkept"], "ground": {}, "eom": {}}
    eg = [p["e_ccsdt"] for p in trunc]
    x = pkg.xfno_extrapolate(f, eg)
    summary["ground"] = {"fno_err_eh": [e - full["e_ccsdt"] for e in eg], "xfno_err_eh": x - full["e_ccsdt"]}
    for var in VARIANTS:
        ref = np.asarray(full["eom"][var]["energies"])
        rows = np.asarray([p["eom"][var]["energies"] for p in trunc])
        xf = np.asarray([pkg.xfno_extrapolate(f, rows[:, k]) for k in range(rows.shape[1])])
        summary["eom"][var] = {"fno_99.9_err_eh": [float(e) for e in rows[0] - ref],
                               "max_abs_fno_err_eh": [float(np.max(np.abs(r - ref))) for r in rows],
                               "xfno_err_eh": [float(e) for e in xf - ref],
                               "max_abs_xfno_err_eh": float(np.max(np.abs(xf - ref)))}
    emit(summary)


# learned-guess check: (electrons, orbitals, kept natural virtuals, variant)
# of the evaluation systems (12-16 electrons, 30-40 kept virtuals), 8 roots
# each
GC_SYSTEMS = ((16, 80, 36, "dip"), (12, 60, 30, "dip"), (16, 80, 32, "dea"), (12, 60, 30, "dea"))
GC_ROOTS = 8


def run_guess_check(args):
    """Davidson starts at a matched 1e-6 Eh target: the guess network is
    trained on --gc-train seeded systems of 6-10 electrons (outside every
    timed region; with --gc-diag-samples the preconditioner target is the
    exact diagonal at that many sampled elements per space, and at most
    --gc-max-samples samples are kept), then DIP and DEA on 12 and 16
    electrons with 30-36 kept natural virtuals, 8 roots each, BF16x3
    products throughout (residual 1e-6), from the diagonal, Koopmans and
    learned starts. Reports products, iterations, wall-clock seconds and the
    largest root difference to the Koopmans solve; one JSON line per
    finished solve, then a summary line."""
    import paper_2509_14157_gb300 as pkg
    from paper_2509_14157_gb300 import learned
    import synth

    def emit(d):
        print(json.dumps(d), flush=True)

    t0 = time.perf_counter()
    X, T, W, info = learned.training_set(learned.seeded_training_systems(args.gc_train, electrons=(6, 8, 10)),
                                         list(VARIANTS), NROOTS, diag_samples=args.gc_diag_samples,
                                         max_samples=args.gc_max_samples, workers=args.gc_workers)
    t_data = time.perf_counter() - t0
    epochs = args.gc_epochs
    net, hist = learned.train_guess_model(X, T, W, epochs=epochs, batch=2048 if X.shape[0] < 10 ** 6 else 8192)
    training = {"seconds": time.perf_counter() - t0, "data_seconds": t_data, "samples": int(X.shape[0]),
                "systems": len(set(i[0] for i in info)), "requested_systems": args.gc_train,
                "diag_samples_per_space": args.gc_diag_samples, "epochs": epochs, "workers": args.gc_workers,
                "first_loss": float(hist[0]), "final_loss": float(hist[-1])}
    emit({"part": "training", **training})
    summary = {"mode": "guess_check", "roots": GC_ROOTS, "precision": "mixed (BF16x3), residual 1e-6",
               "training": training, "data": "synthetic", "systems": []}
    for ne, norb, nkeep, var in GC_SYSTEMS:
        h, eri = synth.hamiltonian(ne, norb, seed=0)
        ctx = pkg.Context(0)
        fi = ctx.fno_truncate(h, eri, ne // 2, 0.0, nkeep=nkeep)
        o, v, _ = ctx.dims()
        cc = ctx.ccsdt_solve(precision="mixed", switch_tol=1e-6)
        ctx.set_guess_model(net)
        res = {}
        for guess in ("diagonal", "koopmans", "learned"):
            t0 = time.perf_counter()
            r = ctx.eom_solve(var, GC_ROOTS, guess=guess, precision="mixed", switch_tol=0.0, tol_res=1e-6,
                              tol_e=1e-8)
            res[guess] = {"seconds": time.perf_counter() - t0, "sigma_calls": r["sigma_calls"], "iters": r["iters"],
                          "converged": r["converged"], "guess_used": r["guess_used"],
                          "energies": [float(x) for x in r["energies"]]}
            emit({"part": "eom", "electrons": ne, "variant": var, "guess": guess, **res[guess]})
        ref = np.asarray(res["koopmans"]["energies"])
        for guess in res:
            res[guess]["max_root_diff_to_koopmans_eh"] = float(np.max(np.abs(np.asarray(res[guess]["energies"]) - ref)))
        summary["systems"].append({"electrons": ne, "orbitals": norb, "nkeep": nkeep, "nkept": fi["nkept"],
                                   "o": o, "v": v, "variant": var, "ccsdt_converged": cc["converged"],
                                   "solves": res})
        ctx.set_guess_model(None)
        ctx.close()
    net.close()
    emit(summary)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fnocc", choices=["fnocc", "reference"])
    ap.add_argument("--threshold", type=float, default=THRESHOLD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_tf32"],
                    help="mixed: BF16 three-slice tensor-core contractions, then FP64 refinement; "
                         "mixed_tf32: TF32 two-slice")
    ap.add_argument("--guess", default="koopmans", choices=["koopmans", "learned"],
                    help="learned: Davidson start and preconditioner from a network trained first (untimed)")
    ap.add_argument("--no-mixed-learned", action="store_true",
                    help="skip the mixed-precision + learned-guess arm of the default run")
    ap.add_argument("--batch", action="store_true",
                    help="many uneven independent systems: batched (one stream per worker) vs one at a time")
    ap.add_argument("--batch-large", action="store_true",
                    help="with --batch: 32 systems of 6-14 electrons and 20-40 kept virtuals, IP/EA x 4 roots, "
                         "BF16x3 with FP64 refinement")
    ap.add_argument("--guess-check", action="store_true",
                    help="diagonal vs Koopmans vs learned Davidson start at a matched 1e-6 Eh target, 8 roots of "
                         "DIP (16 electrons) and DEA (12 electrons)")
    ap.add_argument("--xfno-check", action="store_true",
                    help="FNO at the paper's three OCCT thresholds and untruncated, CCSDT and 4 roots of every "
                         "variant each; FNO and XFNO errors against the untruncated energies")
    ap.add_argument("--gc-train", type=int, default=12,
                    help="with --guess-check: number of seeded training systems")
    ap.add_argument("--gc-diag-samples", type=int, default=None,
                    help="with --guess-check: exact-diagonal targets at this many sampled elements per space "
                         "(default: every element)")
    ap.add_argument("--gc-max-samples", type=int, default=None,
                    help="with --guess-check: keep at most this many training samples (seeded draw)")
    ap.add_argument("--gc-epochs", type=int, default=30, help="with --guess-check: training epochs")
    ap.add_argument("--gc-workers", type=int, default=1,
                    help="with --guess-check: host threads (one context each) building the training set")
    ap.add_argument("--precision-check", action="store_true",
                    help="split-product accuracy and speed on 16 electrons / 80 orbitals, IP/EA/DIP x 6 roots")
    ap.add_argument("--pc-variants", default=None,
                    help="with --precision-check: comma-separated variants (default ip,ea,dip; dea fits on the "
                         "device at this size, its FP64 solve takes about a quarter of an hour)")
    ap.add_argument("--pc-kinds", default=None,
                    help="with --precision-check: comma-separated split kinds (default mixed,mixed_tf32)")
    ap.add_argument("--solve-only", default=None, choices=list(VARIANTS) + ["ee"],
                    help="FNO, CCSDT and one Davidson solve of this variant (4 roots) at the workload's size")
    ap.add_argument("--warm", type=int, default=2,
                    help="with --sigma-only: warm products before the timed one (tile-shape timing needs one "
                         "per candidate)")
    ap.add_argument("--tile-shape", type=int, default=-1,
                    help="with --sigma-only: force one grouped-GEMM tile shape (fnocc_set_tile_shape)")
    ap.add_argument("--mid", action="store_true",
                    help="with --sigma-only: 12 electrons / 60 orbitals, FNO 1e-4 (o = 12, v = 34)")
    ap.add_argument("--large", action="store_true",
                    help="with --sigma-only / --solve-only: the larger system (16 electrons / 80 orbitals, FNO "
                         "1e-6: 41 kept natural virtuals, o = 16, v = 82), 6 roots; mixed solves run CCSDT mixed")
    ap.add_argument("--left", action="store_true",
                    help="with --sigma-only / --solve-only: the left product / left eigenvectors")
    ap.add_argument("--sigma-only", default=None, choices=list(VARIANTS) + ["ee"],
                    help="one sigma product at the workload's size (profiling case)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.sigma_only:
        return run_sigma_only(args)
    if args.solve_only:
        return run_solve_only(args)
    if args.batch:
        return run_batch(args)
    if args.precision_check:
        return run_precision_check(args)
    if args.guess_check:
        return run_guess_check(args)
    if args.xfno_check:
        return run_xfno_check(args)

    import torch
    import torch.distributed as dist
    import paper_2509_14157_gb300 as pkg
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    seed = replica_seed(rank)
    h, eri = synth.hamiltonian(NE, NORB, seed=seed)
    nocc = NE // 2
    # end-to-end inputs live in pinned host memory (page-locked copies)
    h_pin = torch.from_numpy(h).pin_memory().numpy()
    eri_pin = torch.from_numpy(eri).pin_memory().numpy()
    h_dev = torch.from_numpy(h).to(dev)
    eri_dev = torch.from_numpy(eri).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)  # 512 MB > L2
    torch.cuda.synchronize()
    ctx = pkg.Context(local, stream.cuda_stream)

    counts = {"cc_iters": 0, "sigma": {}, "detail": {}, "flops_per_sigma": {}}

    # mixed kinds: split products throughout the Davidson solves, converged to
    # the 1e-6 Eh accuracy target (no FP64 refinement sweep); CCSDT refines in FP64
    eom_kw = (dict(precision=args.precision, switch_tol=0.0, tol_res=1e-6, tol_e=1e-8, guess="koopmans")
              if args.precision != "fp64" else dict(precision="fp64", guess="koopmans"))
    guess_net = {}

    def train_guess():
        """The guess network, trained once (outside every timed region) on
        small seeded systems solved by the library itself."""
        if "net" not in guess_net:
            from paper_2509_14157_gb300 import learned
            t0 = time.perf_counter()
            X, T, W, info = learned.training_set(learned.seeded_training_systems(12), list(VARIANTS), NROOTS,
                                                 device=local)
            net, hist = learned.train_guess_model(X, T, W, epochs=30, batch=2048, device=local)
            guess_net.update(net=net, seconds=time.perf_counter() - t0, samples=int(X.shape[0]),
                             systems=len(set(i[0] for i in info)), final_loss=float(hist[-1]))
        ctx.set_guess_model(guess_net["net"])
        return guess_net

    if args.guess == "learned":
        train_guess()
        eom_kw = dict(eom_kw, guess="learned")

    def step(device_inputs, prec=args.precision, kw=eom_kw):
        t0 = time.perf_counter()
        if device_inputs:
            ctx.fno_truncate_dev(h_dev.data_ptr(), eri_dev.data_ptr(), NORB, nocc, args.threshold)
        else:
            ctx.fno_truncate(h_pin, eri_pin, nocc, args.threshold)
        counts["fno_seconds"] = round(time.perf_counter() - t0, 4)
        f0 = ctx.flops
        res = ctx.ccsdt_solve(precision=prec)
        if not res["converged"]:
            raise RuntimeError("CCSDT did not converge")
        counts["cc_iters"] = res["iters"]
        counts["ccsdt_seconds"] = round(res["seconds"], 4)
        counts["ccsdt_seconds_per_iter"] = round(res["seconds_per_iter"], 5)
        counts["flops_per_residual"] = (ctx.flops - f0) / max(1, res["iters"])
        out = {}
        for var in VARIANTS:
            f0 = ctx.flops
            r = ctx.eom_solve(var, NROOTS, **kw)
            counts["flops_per_sigma"][var] = (ctx.flops - f0) / max(1, r["sigma_calls"])
            if not r["converged"]:
                raise RuntimeError("%s-EOM did not converge" % var)
            counts["sigma"][var] = r["sigma_calls"]
            counts["detail"][var] = {"iters": r["iters"], "res_max": r["res_max"],
                                     "complex_roots": r["complex_roots"], "seconds": round(r["seconds"], 3),
                                     "seconds_per_iter": round(r["seconds_per_iter"], 5)}
            out[var] = r["energies"]
        return res, out

    for _ in range(args.warmup):
        step(True)
    fp64_fma, fp64_dmma, fp64_basis = measured_fp64_peak(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    launches0, flops0 = ctx.launches, ctx.flops
    times = []
    last_roots = {}
    for k in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if k == args.steps - 1:
            torch.cuda.nvtx.range_push("step")  # the last timed step, for launch lists
        e0.record(stream)
        _, last_roots["fp64"] = step(True)
        e1.record(stream)
        if k == args.steps - 1:
            torch.cuda.nvtx.range_pop()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    launches = ctx.launches - launches0
    flops = ctx.flops - flops0
    # per-kernel timing: one more step of the same work with CUDA events
    # around every contraction launch (plain launches: the timed steps replay
    # the products' launch sequences as graphs, which per-launch events would
    # break up)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(-1)
    step(True)
    torch.cuda.synchronize()
    paths = {}
    for pid, name in ctx.PROFILE_PATHS.items():
        ms_, fl_, n_ = ctx.profile_read(pid)
        paths[name] = {"ms": ms_, "flops": fl_, "launches": n_}
    ctx.profile(False)
    dominant = max(paths, key=lambda k: paths[k]["ms"])
    gemm_ms, gemm_flops, gemm_n = paths[dominant]["ms"], paths[dominant]["flops"], paths[dominant]["launches"]
    clocks = sampler.stop()
    total = sum(times)
    total = max_over_ranks(total, world, dev)
    if world > 1:
        dist.barrier()
    # end to end: host buffers through the C ABI, copies and read-back inside
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(False)
        e2e_times.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_times)
    e2e_total = max_over_ranks(e2e_total, world, dev)
    # solver statistics of the timed path (the arms below reuse `counts`)
    path_counts = copy.deepcopy(counts)
    accuracy = None
    if args.precision != "fp64":
        # every root against the same solve in FP64 (outside the timed region)
        _, mixed_e = step(True)
        _, ref_e = step(True, "fp64", dict(precision="fp64"))
        accuracy = {"target_eh": 1e-6, "reference": "FP64 path, same inputs",
                    "max_abs_err_eh": {v: float(np.max(np.abs(np.asarray(mixed_e[v]) - np.asarray(ref_e[v]))))
                                       for v in VARIANTS},
                    "per_root_err_eh": {v: [float(x) for x in np.asarray(mixed_e[v]) - np.asarray(ref_e[v])]
                                        for v in VARIANTS}}
    mixed_learned = None
    if args.precision == "fp64" and args.guess == "koopmans" and not args.no_mixed_learned:
        # the BF16x3 + learned-guess arm on the same inputs, at the 1e-6 Eh target
        info = train_guess()
        # split products until every residual norm is below 1e-5, then FP64
        # refinement sweeps to residual 1e-6 / |d omega| 1e-8
        kw = dict(precision="mixed", switch_tol=1e-5, tol_res=1e-6, tol_e=1e-8, guess="learned")
        _, ref_e = step(True)
        step(True, "mixed", kw)
        ml_times = []
        ml_flops0 = ctx.flops
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, ml_e = step(True, "mixed", kw)
            e1.record(stream)
            e1.synchronize()
            ml_times.append(e0.elapsed_time(e1) / 1e3)
        ml_total = sum(ml_times)
        ml_total = max_over_ranks(ml_total, world, dev)
        ml_flops = ctx.flops - ml_flops0
        # per-kernel timing of the arm: one profiled step (plain launches)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(-1)
        step(True, "mixed", kw)
        torch.cuda.synchronize()
        ml_paths = {}
        for pid, name in ctx.PROFILE_PATHS.items():
            ms_, fl_, n_ = ctx.profile_read(pid)
            ml_paths[name] = {"ms": ms_, "flops": fl_, "launches": n_}
        ctx.profile(False)
        mixed_learned = {
            "value": ml_total / (len(VARIANTS) * args.steps * world), "unit": "s",
            "tflops": ml_flops * world / ml_total / 1e12 if ml_total > 0 else None,
            "ms_per_step": 1e3 * ml_total / args.steps,
            "config": "BF16x3 products until every Davidson residual is below 1e-5, then FP64 refinement "
                      "sweeps to residual 1e-6 and |d omega| 1e-8; learned start and preconditioner; CCSDT "
                      "BF16x3 then FP64 below 1e-6",
            "vs_oracle": oracle_root_errors(ml_e, args.threshold, seed),
            "roofline": split_roofline(ml_paths, ml_total / args.steps),
            "sigma_calls": dict(counts["sigma"]),
            "max_abs_err_eh": {v: float(np.max(np.abs(np.asarray(ml_e[v]) - np.asarray(ref_e[v]))))
                               for v in VARIANTS},
            "target_eh": 1e-6,
            "guess_training": {"seconds": round(info["seconds"], 2), "systems": info["systems"],
                               "samples": info["samples"], "final_loss": info["final_loss"],
                               "workload": "12 seeded systems, 6 or 8 electrons, 10-12 orbitals, 4-6 kept "
                                           "natural virtuals, IP/EA/DIP/DEA x 4 roots"}}
    solves = len(VARIANTS) * args.steps * world
    value = total / solves
    parity = oracle_root_errors(last_roots["fp64"], args.threshold, seed) if args.precision == "fp64" else None
    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None
    traffic = read_traffic()
    if dominant.startswith("k_ggemm_bf16x3"):
        # six BF16 slice products per FP64-equivalent multiply-add
        peak, basis = measured_bf16_peak()
        roof = {"bound": "tensor", "kernel": dominant + " (BF16 mma.sync, 6 slice products)",
                "achieved": 6 * achieved if achieved else None, "peak": peak, "unit": "TFLOP/s",
                "frac": 6 * achieved / peak if achieved else None, "traffic": None, "peak_basis": basis}
    elif dominant.startswith("k_ggemm_tf32x3"):
        # three TF32 slice products per FP64-equivalent multiply-add; TF32 peak =
        # measured BF16 peak x the nominal dense ratio 1.1 / 2.25 PFLOP/s
        peak, basis = measured_bf16_peak()
        peak *= 1.1 / 2.25
        roof = {"bound": "tensor", "kernel": dominant + " (TF32 mma.sync, 3 slice products)",
                "achieved": 3 * achieved if achieved else None, "peak": peak, "unit": "TFLOP/s",
                "frac": 3 * achieved / peak if achieved else None, "traffic": None,
                "peak_basis": basis + " x 1.1/2.25 (nominal TF32/BF16)"}
    else:
        roof = {"bound": "alu", "kernel": dominant + " (FP64 FMA)", "achieved": achieved,
                "peak": fp64_fma, "unit": "TFLOP/s",
                "frac": achieved / fp64_fma if achieved else None,
                "traffic": traffic if dominant == "k_ggemm" else None,
                "peak_basis": fp64_basis, "peak_fp64_dmma_measured": fp64_dmma,
                "peak_derived": FP64_PEAK_DERIVED_TFLOPS,
                "frac_of_derived": achieved / FP64_PEAK_DERIVED_TFLOPS if achieved else None}
    roof.update({"launches": gemm_n, "share_of_step": (gemm_ms / 1e3) / (total / args.steps) if total else None,
                 "measured_on": "one profiled step after the timed ones (CUDA events around every "
                                "contraction launch, plain launches)",
                 "paths": {k: {"ms": round(x["ms"], 3),
                               "tflops": (x["flops"] / x["ms"] / 1e9) if x["ms"] else None,
                               "launches": x["launches"]} for k, x in paths.items()}})
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "bf16x3->f32, f64 refinement",
                  "mixed_tf32": "tf32x3->f32, f64 refinement"}[args.precision],
        "data": "synthetic", "config": dict(config(args.threshold, seed), precision=args.precision),
        "tflops": flops * world / total / 1e12 if total > 0 else None,
        "roofline": roof,
        "e2e": {"value": e2e_total / solves, "unit": "s",
                "h2d_bytes_per_step": int(h.nbytes + eri.nbytes),
                "d2h_bytes_per_step": int(8 * (len(VARIANTS) * NROOTS * 2 + (NORB - nocc)))},
        "gpu_launches": launches, "clocks": clocks,
        **({"parity": parity} if parity else {}),
        **({"accuracy": accuracy} if accuracy else {}),
        **({"mixed_learned": mixed_learned} if mixed_learned else {}),
        **({"guess": "learned", "guess_training": {k: v for k, v in guess_net.items() if k != "net"}}
           if args.guess == "learned" else {}),
        "solver": {"fno_seconds": path_counts["fno_seconds"], "ccsdt_seconds": path_counts["ccsdt_seconds"],
                   "ccsdt_seconds_per_iter": path_counts["ccsdt_seconds_per_iter"],
                   "ccsdt_iters": path_counts["cc_iters"], "sigma_calls": path_counts["sigma"],
                   "eom": path_counts["detail"], "flops_per_residual": path_counts["flops_per_residual"],
                   "flops_per_sigma": path_counts["flops_per_sigma"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.threshold, path_counts)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
