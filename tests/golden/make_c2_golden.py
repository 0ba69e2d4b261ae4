"""Writes tests/golden/c2_oracle.json with the CPU oracle only.

Workload: the 10-electron / 48-orbital seeded synthetic closed-shell
Hamiltonian (synth.hamiltonian(10, 48, seed=0)), natural virtuals kept at
occupation >= 1e-4 (15 of 43 spatial virtuals: o = 10, v = 30 spin
orbitals), the CCSDT ground state converged to max|R| < 1e-12, and the four
lowest roots of IP-, EA-, DIP- and DEA-EOM-CCSDT in their target spin
sectors (Davidson from the Koopmans guess, residual 1e-8, |d omega| 1e-10,
roots counted among principal-weight states).

Every residual (Eq. 6) and product (Eq. 1-4) is the oracle's own sum over
its Wick terms (oracle.wick.evaluate on dense tensors, then oracle.packing);
the only addition is plumbing: the terms of one evaluation are dealt out to
worker processes, each of which sums a disjoint subset and returns the
packed partial sum, and the parent adds the partial sums (only the order of
the additions differs from one process, i.e. rounding). The solvers are the
oracle's (oracle.cc.ccsdt, oracle.eom.eom_ccsdt) with their evaluation
function swapped for this split one.

Stored: FNO quantities, E_corr and iteration count, the packed T1 block, a
seeded sample of packed T2 and T3 elements (index and value) with the 2-norm
of each block, and the roots of every variant.

Run (several hours on 8 cores; the DEA products dominate):
    python tests/golden/make_c2_golden.py [--workers N] [--variants ip,ea,dip,dea]

With --occt F the virtuals are kept by the cumulative-occupation criterion
instead (the shortest prefix of natural occupations reaching the fraction
F, the paper's OCCT thresholds), written to c2_occt<F>_oracle.json: at
F = 0.995, 17 of 43 natural virtuals (o = 10, v = 34), one of the three
truncations the XFNO extrapolation combines.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import cc, eom, fno, packing, wick  # noqa: E402

NE, NORB, THRESHOLD, NROOTS = 10, 48, 1e-4, 4
SAMPLES = 256

_W = {}


def _worker_init(ham_path):
    sys.path.insert(0, ROOT)
    d = np.load(ham_path)
    _W["f"], _W["g"], _W["o"], _W["v"] = d["f"], d["g"], int(d["o"]), int(d["v"])


def _worker_eval(task):
    """task: (amplitude file, [(kind, variant, out_comp, in_comp, term index)])
    -> {out_comp: packed partial sum}."""
    amp_dir, items = task
    amps = {nm[:-4]: np.load(os.path.join(amp_dir, nm), mmap_mode="r")
            for nm in os.listdir(amp_dir) if nm.endswith(".npy")}
    f, g, o, v = _W["f"], _W["g"], _W["o"], _W["v"]
    out = {}
    for kind, variant, oc, ic, k in items:
        if kind == "cc":
            terms = wick.cc_terms(oc)
            nh = np_ = oc
        else:
            terms = wick.eom_terms(variant, oc, ic)
            nh, np_ = wick.EOM_SPACES[variant][oc]
        dense = wick.evaluate((terms[k],), nh, np_, f, g, amps, o, v)
        part = np.atleast_1d(dense).reshape(-1) if nh + np_ == 0 else packing.pack(dense, nh, np_, o, v)
        out[oc] = out.get(oc, 0.0) + part
    return out


class Split:
    """Evaluates a sum over Wick terms across worker processes."""

    def __init__(self, pool, workers, tmpdir):
        self.pool, self.workers, self.tmpdir = pool, workers, tmpdir
        self.calls = 0

    def run(self, items, amps):
        self.calls += 1
        path = os.path.join(self.tmpdir, "amps_%d" % self.calls)
        os.makedirs(path)
        for nm, x in amps.items():
            np.save(os.path.join(path, nm + ".npy"), np.ascontiguousarray(x))
        # largest outputs first, dealt round-robin so that every worker gets a
        # share of the expensive terms
        chunks = [[] for _ in range(self.workers)]
        for j, it in enumerate(items):
            chunks[j % self.workers].append(it)
        parts = self.pool.map(_worker_eval, [(path, c) for c in chunks if c])
        for nm in os.listdir(path):
            os.remove(os.path.join(path, nm))
        os.rmdir(path)
        acc = {}
        for p in parts:
            for oc, x in p.items():
                acc[oc] = acc.get(oc, 0.0) + x
        return acc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--variants", default="ip,ea,dip,dea")
    ap.add_argument("--occt", type=float, default=None,
                    help="keep virtuals by cumulative occupation fraction instead of the 1e-4 threshold")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    here = os.path.dirname(os.path.abspath(__file__))
    if args.occt is None:
        tag, crit, thr = "", "abs", THRESHOLD
        workload = "10 electrons, 48 spatial orbitals, seed 0, FNO occupation threshold 1e-4"
    else:
        tag, crit, thr = "_occt%g" % (args.occt * 1000), "occt", args.occt
        workload = ("10 electrons, 48 spatial orbitals, seed 0, FNO by cumulative occupation fraction %g"
                    % args.occt)
    if args.out is None:
        args.out = os.path.join(here, "c2%s_oracle.json" % tag)
    t0 = time.time()
    h, eri = synth.hamiltonian(NE, NORB, seed=0)
    act = fno.fno_truncate(h, eri, NE // 2, thr, criterion=crit)
    f, g, o, v = act["f"], act["g"], act["o"], act["v"]
    out = dict(workload=workload, criterion=crit, threshold=thr,
               e_rhf=act["e_rhf"], e_mp2=act["e_mp2"], nkept=int(act["nkept"]),
               kept_fraction=act["kept_fraction"], e_ref=act["e_ref"], o=o, v=v, eom={})
    if os.path.exists(args.out):  # resume: keep what an earlier run finished
        old = json.load(open(args.out))
        if old.get("o") == o and old.get("v") == v:
            out = old
            out.setdefault("eom", {})
    # one BLAS thread per worker: the workers already use the cores
    for var_name in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var_name] = "1"
    tmpdir = tempfile.mkdtemp(prefix="c2golden_", dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
    ham_path = os.path.join(tmpdir, "ham.npz")
    np.savez(ham_path, f=f, g=g, o=o, v=v)
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers, initializer=_worker_init, initargs=(ham_path,)) as pool:
        split = Split(pool, args.workers, tmpdir)
        cc_items = [("cc", None, r, 0, k) for r in (3, 2, 1) for k in range(len(wick.cc_terms(r)))]

        def residuals(f_, g_, o_, v_, t1, t2, t3):
            acc = split.run(cc_items, {"t1": t1, "t2": t2, "t3": t3})
            return [packing.unpack(acc[r], r, r, o_, v_) for r in (1, 2, 3)]

        # converged amplitudes kept outside the repository, so that a rerun
        # can resume with the EOM part
        amp_path = os.path.join(tempfile.gettempdir(), "fnocc_c2%s_oracle_amplitudes.npz" % tag)
        if "e_ccsdt_corr" in out and os.path.exists(amp_path):
            d = np.load(amp_path)
            t1, t2, t3 = (packing.unpack(d["t%d" % r], r, r, o, v) for r in (1, 2, 3))
        else:
            cc.residuals = residuals  # the oracle's solver with the split evaluation
            res = cc.ccsdt(f, g, o, v, tol_res=1e-12, tol_e=1e-13)
            t1, t2, t3 = res["t1"], res["t2"], res["t3"]
            pk = {"t%d" % r: packing.pack(x, r, r, o, v) for r, x in ((1, t1), (2, t2), (3, t3))}
            np.savez(amp_path, **pk)
            rng = np.random.default_rng(2025)
            out.update(e_ccsdt_corr=res["e_corr"], ccsdt_iters=res["iters"], ccsdt_converged=bool(res["converged"]),
                       ccsdt_res_max=float(res["res"]), t1=[float(x) for x in pk["t1"]],
                       t_norms={k: float(np.linalg.norm(x)) for k, x in pk.items()}, t_samples={})
            for r in (2, 3):
                idx = np.sort(rng.choice(len(pk["t%d" % r]), size=SAMPLES, replace=False))
                out["t_samples"]["t%d" % r] = {"index": [int(i) for i in idx],
                                               "value": [float(pk["t%d" % r][i]) for i in idx]}
            json.dump(out, open(args.out, "w"), indent=1)
            print("ccsdt", res["e_corr"], res["iters"], "%.0f s" % (time.time() - t0), flush=True)
        for var in args.variants.split(","):
            if var in out["eom"]:
                continue
            items = [("eom", var, oc, ic, k) for oc in (2, 1, 0) for ic in range(3)
                     for k in range(len(wick.eom_terms(var, oc, ic)))]

            def sigma_packed(variant, f_, g_, o_, v_, t1_, t2_, t3_, vec, _items=items):
                rs = eom.split(variant, o_, v_, vec)
                acc = split.run(_items, {"t1": t1_, "t2": t2_, "t3": t3_, "r1": rs[0], "r2": rs[1], "r3": rs[2]})
                return np.concatenate([np.asarray(acc.get(oc, np.zeros(n)), dtype=float)
                                       for oc, n in enumerate(eom.sizes(variant, o_, v_))])

            eom.sigma_packed = sigma_packed  # the oracle's Davidson with the split evaluation
            c0 = split.calls
            r = eom.eom_ccsdt(var, f, g, o, v, t1, t2, t3, NROOTS, guess="koopmans")
            out["eom"][var] = dict(omega=[float(x) for x in r["omega"]], converged=bool(r["converged"]),
                                   iters=int(r["iters"]), products=split.calls - c0,
                                   res=[float(x) for x in r["res"]])
            json.dump(out, open(args.out, "w"), indent=1)
            print(var, r["omega"], r["converged"], "%.0f s" % (time.time() - t0), flush=True)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
