"""Every tile shape of the grouped contraction kernel against the oracle.

The library normally picks one shape per contraction step (least padded work
per busy SM, large FP64 steps timed once), so a shape that no step happens to
pick would otherwise never run. Here each shape is forced for every grouped
step (fnocc_set_tile_shape) of one IP and one DEA product, and of one CCSDT
residual, on a random non-canonical Hamiltonian with 6 occupied and 14
virtual spin orbitals: several tiles with ragged tails for the small shapes,
one ragged tile for the large ones.

Tolerances: FP64 shapes 1e-10 max-abs (the FP64 path's bound); split-product
shapes run in their own arithmetic (BF16 three-slice or TF32 two-slice, FP32
accumulation; on mma.sync, and BF16 three-slice also on the tcgen05 tensor
cores with a tensor-memory accumulator) and are held to the relative product
bounds of the mixed path (2e-6 and 1e-5 of the largest element).
"""
import math

import numpy as np
import pytest

import synth
from oracle import cc, eom, fno, packing, wick

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-10
MIXED_TOL = {"mixed": 2e-6, "mixed_tf32": 1e-5}


@pytest.fixture(scope="module")
def pkg():
    import paper_2509_14157_gb300 as p
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def spin_masked(nh, np_, o, v, seed, scale, ms2=0):
    x = synth.random_packed(math.comb(o, nh) * math.comb(v, np_), seed, scale)
    return x * synth.packed_ms_mask(nh, np_, o, v, ms2)


@pytest.fixture(scope="module")
def system(pkg):
    nocc, n = 3, 10
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 61)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    t = [spin_masked(r, r, o, v, 500 + r, 0.05) for r in (1, 2, 3)]
    td = [packing.unpack(t[r - 1], r, r, o, v) for r in (1, 2, 3)]
    ref = {"residual": cc.residuals_packed(ham["f"], ham["g"], o, v, *t)}
    vecs = {}
    for variant in ("ip", "dea"):
        ms2 = eom.SECTOR_MS2[variant]
        x = np.concatenate([spin_masked(nh, np_, o, v, 510 + k, 0.3, ms2)
                            for k, (nh, np_) in enumerate(wick.EOM_SPACES[variant])])
        vecs[variant] = x
        ref[variant] = eom.sigma_packed(variant, ham["f"], ham["g"], o, v, *td, x)
    ctx = pkg.Context(0)
    ctx.set_mo_hamiltonian(h, eri, nocc)
    yield ctx, t, vecs, ref
    ctx.close()


def _shapes(pkg):
    count, first_mixed = pkg.tile_shapes()
    return count, first_mixed


def test_shape_table(pkg):
    count, first_mixed = _shapes(pkg)
    assert first_mixed == 19 < count
    kinds = [pkg.tile_shape_kind(k) for k in range(count)]
    assert kinds[:first_mixed] == [0] * first_mixed
    assert 1 in kinds and 2 in kinds and 3 in kinds and kinds == sorted(kinds)
    assert pkg.tile_shape_kind(count) == -1


@pytest.mark.parametrize("shape", range(19))
def test_fp64_shape_products(pkg, system, shape):
    count, first_mixed = _shapes(pkg)
    if shape >= first_mixed:
        pytest.skip("not an FP64 shape")
    ctx, t, vecs, ref = system
    ctx.set_precision("fp64")
    ctx.set_tile_shape(shape)
    try:
        ctx.set_amplitudes(*t)
        for variant in ("ip", "dea"):
            got = ctx.eom_sigma(variant, vecs[variant])
            assert np.max(np.abs(got - ref[variant])) < AMP_TOL, (shape, variant)
        res, _ = ctx.ccsdt_residual(*t)
        for a, b in zip(res, ref["residual"]):
            assert np.max(np.abs(a - b)) < AMP_TOL, shape
    finally:
        ctx.set_tile_shape(-1)


@pytest.mark.parametrize("kind", ["mixed", "mixed_tf32"])
def test_split_shape_products(pkg, system, kind):
    count, first_mixed = _shapes(pkg)
    ctx, t, vecs, ref = system
    ctx.set_precision(kind)
    try:
        for shape in range(first_mixed, count):
            if kind == "mixed_tf32" and pkg.tile_shape_kind(shape) >= 2:
                continue  # tcgen05 tiles run BF16x3 only
            ctx.set_tile_shape(shape)
            ctx.set_amplitudes(*t)
            for variant in ("ip", "dea"):
                got = ctx.eom_sigma(variant, vecs[variant])
                scale = np.max(np.abs(ref[variant]))
                assert np.max(np.abs(got - ref[variant])) < MIXED_TOL[kind] * scale, (shape, variant)
            res, _ = ctx.ccsdt_residual(*t)
            for a, b in zip(res, ref["residual"]):
                if b.size:
                    assert np.max(np.abs(a - b)) < MIXED_TOL[kind] * max(np.max(np.abs(b)), 1e-30), shape
    finally:
        ctx.set_tile_shape(-1)
        ctx.set_precision("fp64")


def test_bad_shape_rejected(pkg, system):
    ctx = system[0]
    count, _ = _shapes(pkg)
    for bad in (-2, count):
        with pytest.raises(pkg.FnoccError):
            ctx.set_tile_shape(bad)
