"""Mixed precision (split products on the tensor cores, FP32 accumulation)
against the FP64 path of the same library and the oracle, for both split
kinds:

  * mixed (BF16 three-slice): operands truncated to FP32 (2^-23 relative
    each), slices exact, the dropped products below 3 * 2^-24: about 3e-7 per
    product. One residual / sigma evaluation within 2e-6 of the largest
    element; solves kept in mixed precision throughout within 1e-6 Eh per
    root of the FP64 oracle, the accuracy target of the mixed path.
  * mixed_tf32 (TF32 two-slice): the low slice rounded to 11 bits (2^-22 per
    operand) and lo * lo dropped (2^-22) on top of the FP32 truncation: about
    1e-6 per product, three times the BF16 split; bounds scaled by 5 (1e-5 of
    the largest element, 5e-6 Eh per root).
  * solves that switch to FP64 refinement reproduce the FP64 energies to the
    FP64 tolerances (1e-9 Eh) with either kind.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import eom, wick

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def pkg():
    import paper_2509_14157_gb300 as p
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


@pytest.fixture(scope="module")
def c2(pkg):
    h, eri = synth.hamiltonian(10, 48, seed=0)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, 5, 1e-4)
    yield ctx
    ctx.close()


KINDS = ["mixed", "mixed_tf32"]
PRODUCT_TOL = {"mixed": 2e-6, "mixed_tf32": 1e-5}
ROOT_TOL_EH = {"mixed": 1e-6, "mixed_tf32": 5e-6}


def spin_masked(nh, np_, o, v, seed, scale, ms2=0):
    x = synth.random_packed(math.comb(o, nh) * math.comb(v, np_), seed, scale)
    return x * synth.packed_ms_mask(nh, np_, o, v, ms2)


@pytest.mark.parametrize("kind", KINDS)
def test_mixed_residual_relative_error(c2, kind):
    o, v, _ = c2.dims()
    t = [spin_masked(r, r, o, v, 500 + r, 0.02) for r in (1, 2, 3)]
    c2.set_precision("fp64")
    ref, e_ref = c2.ccsdt_residual(*t)
    c2.set_precision(kind)
    got, e = c2.ccsdt_residual(*t)
    c2.set_precision("fp64")
    for a, b in zip(got, ref):
        rel = np.max(np.abs(a - b)) / np.max(np.abs(b))
        assert 0 < rel < PRODUCT_TOL[kind], rel  # > 0: the split path really ran
    assert abs(e - e_ref) < 1e-6


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea"])
def test_mixed_sigma_relative_error(c2, variant, kind):
    o, v, _ = c2.dims()
    c2.set_amplitudes(*[spin_masked(r, r, o, v, 600 + r, 0.02) for r in (1, 2, 3)])
    ms2 = eom.SECTOR_MS2[variant]
    x = np.concatenate([spin_masked(nh, np_, o, v, 70 + k, 0.3, ms2)
                        for k, (nh, np_) in enumerate(wick.EOM_SPACES[variant])])
    c2.set_precision("fp64")
    ref = c2.eom_sigma(variant, x)
    c2.set_precision(kind)
    got = c2.eom_sigma(variant, x)
    c2.set_precision("fp64")
    rel = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert 0 < rel < PRODUCT_TOL[kind], rel


@pytest.mark.parametrize("kind", KINDS)
def test_mixed_solves_against_fp64_and_oracle(pkg, kind):
    """6 electrons / 10 orbitals (FNO 1e-4): refined mixed solves equal the
    oracle to 1e-9 Eh; mixed-only solves stay within the kind's bound per
    root."""
    gold = json.load(open(os.path.join(HERE, "golden", "c1_oracle.json")))
    h, eri = synth.hamiltonian(6, 10, seed=0)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, 3, 1e-4)
    res = ctx.ccsdt_solve(precision=kind, switch_tol=1e-6)
    assert res["converged"] and res["iters_mixed"] > 0
    assert abs(res["e_corr"] - gold["e_ccsdt_corr"]) < 1e-9
    for variant, ent in gold["eom"].items():
        ref = np.array(ent["omega"])
        r = ctx.eom_solve(variant, len(ref), precision=kind, switch_tol=1e-5)
        assert r["converged"] and r["sigma_calls_mixed"] > 0
        assert np.max(np.abs(r["omegas"] - ref)) < 1e-9, variant
        m = ctx.eom_solve(variant, len(ref), precision=kind, switch_tol=0.0, tol_res=1e-6, tol_e=1e-8)
        assert np.max(np.abs(m["omegas"] - ref)) < ROOT_TOL_EH[kind], (variant, m["omegas"] - ref)
    ctx.close()
