"""Writes tests/golden/c1_oracle.json with the CPU oracle only.

Workload: the 6-electron / 10-orbital seeded synthetic closed-shell
Hamiltonian (synth.hamiltonian(6, 10, seed=0)), natural virtuals kept at
occupation >= 1e-4, CCSDT ground state, and the three lowest roots of each
EOM-CCSDT variant in its target spin sector (Davidson, diagonal guess).

Run: python tests/golden/make_golden.py   (from the repository root)
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import cc, eom, fno  # noqa: E402


def main():
    t0 = time.time()
    h, eri = synth.hamiltonian(6, 10, seed=0)
    act = fno.fno_truncate(h, eri, 3, 1e-4)
    f, g, o, v = act["f"], act["g"], act["o"], act["v"]
    res = cc.ccsdt(f, g, o, v)
    out = dict(
        workload="6 electrons, 10 spatial orbitals, seed 0, FNO occupation threshold 1e-4",
        e_rhf=act["e_rhf"], e_mp2=act["e_mp2"], nkept=int(act["nkept"]),
        kept_fraction=act["kept_fraction"], occ=[float(x) for x in act["occ"]],
        e_ref=act["e_ref"], e_ccsdt_corr=res["e_corr"], ccsdt_iters=res["iters"], eom={})
    print("ccsdt", res["e_corr"], time.time() - t0, flush=True)
    for var in ("ip", "ea", "dip", "dea"):
        r = eom.eom_ccsdt(var, f, g, o, v, res["t1"], res["t2"], res["t3"], 3, guess="diagonal")
        out["eom"][var] = dict(omega=[float(x) for x in r["omega"]], converged=bool(r["converged"]),
                               iters=int(r["iters"]))
        print(var, r["omega"], r["converged"], time.time() - t0, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
