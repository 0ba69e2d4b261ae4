"""The stored oracle fixtures of the benchmarked system (tests/golden/,
written by make_c2_golden.py) against a fresh run of the oracle's FNO step
(CPU): the truncation each fixture records and the sizes of what it stores
must be the oracle's, so that the GPU tests compare with the workload they
name."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import fno

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURES = {"c2_oracle.json": ("abs", 1e-4), "c2_occt995_oracle.json": ("occt", 0.995)}


@pytest.fixture(scope="module")
def c2_hamiltonian():
    return synth.hamiltonian(10, 48, seed=0)


@pytest.mark.parametrize("name", sorted(FIXTURES))
def test_fixture_matches_oracle_fno(c2_hamiltonian, name):
    path = os.path.join(HERE, "golden", name)
    if not os.path.exists(path):
        pytest.skip("fixture not written")
    gold = json.load(open(path))
    crit, thr = FIXTURES[name]
    h, eri = c2_hamiltonian
    act = fno.fno_truncate(h, eri, 5, thr, criterion=crit)
    assert gold["o"] == act["o"] and gold["v"] == act["v"] and gold["nkept"] == act["nkept"]
    for key in ("e_rhf", "e_mp2", "kept_fraction", "e_ref"):
        assert abs(gold[key] - act[key]) < 1e-10, key
    o, v = act["o"], act["v"]
    assert len(gold["t1"]) == o * v
    sizes = {"t2": math.comb(o, 2) * math.comb(v, 2), "t3": math.comb(o, 3) * math.comb(v, 3)}
    for r, n in sizes.items():
        idx = np.array(gold["t_samples"][r]["index"])
        assert idx.size == len(gold["t_samples"][r]["value"]) and np.all((idx >= 0) & (idx < n))
        assert np.all(np.diff(idx) > 0)
    assert gold["ccsdt_converged"] and gold["ccsdt_res_max"] < 1e-12
    for var, ent in gold["eom"].items():
        assert ent["converged"] and len(ent["omega"]) == 4, var
        assert np.all(np.diff(ent["omega"]) >= 0), var
