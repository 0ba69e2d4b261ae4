"""Graph replay of the EOM products' launch sequences (fnocc_set_graphs).

Replay runs the same kernels with the same launch parameters in the same
order as the plain launches, so the products must agree bitwise, for every
variant and direction, in FP64 and in the BF16x3 split arithmetic; a
captured graph follows new amplitudes (recaptured), counts its launches
like the plain path, and a Davidson solve gives the same roots with and
without it.
"""
import math

import numpy as np
import pytest

import synth
from oracle import eom, wick

pytestmark = pytest.mark.gpu


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


def vector(variant, o, v, seed):
    ms2 = eom.SECTOR_MS2[variant]
    return np.concatenate([spin_masked(nh, np_, o, v, seed + k, 0.3, ms2)
                           for k, (nh, np_) in enumerate(wick.EOM_SPACES[variant])])


@pytest.fixture(scope="module")
def ctx(pkg):
    h, eri = synth.random_symmetric_mo_hamiltonian(10, 81)
    c = pkg.Context(0)
    c.set_mo_hamiltonian(h, eri, 3)
    o, v, _ = c.dims()
    c.set_amplitudes(*[spin_masked(r, r, o, v, 600 + r, 0.05) for r in (1, 2, 3)])
    yield c
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_replay_is_bitwise_plain(ctx, variant, precision):
    o, v, _ = ctx.dims()
    ctx.set_precision(precision)
    xs = [vector(variant, o, v, s) for s in (700, 710, 720)]
    for left in (False, True):
        product = ctx.eom_left_sigma if left else ctx.eom_sigma
        ctx.set_graphs(False)
        product(variant, xs[0])  # cached pieces valid, tile shapes settled
        ref = [product(variant, x) for x in xs]
        n0 = ctx.launches
        product(variant, xs[0])
        plain_launches = ctx.launches - n0
        ctx.set_graphs(True)
        got = [product(variant, x) for x in xs]  # capture on the first, replay on the others
        n0 = ctx.launches
        product(variant, xs[1])
        assert ctx.launches - n0 == plain_launches
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), (variant, precision, left)
    ctx.set_precision("fp64")


def test_replay_follows_new_amplitudes(pkg):
    h, eri = synth.random_symmetric_mo_hamiltonian(8, 83)
    c = pkg.Context(0)
    c.set_mo_hamiltonian(h, eri, 2)
    o, v, _ = c.dims()
    x = vector("ea", o, v, 730)
    out = []
    for seed in (800, 810):
        t = [spin_masked(r, r, o, v, seed + r, 0.05) for r in (1, 2, 3)]
        c.set_graphs(False)
        c.set_amplitudes(*t)
        plain = c.eom_sigma("ea", x)
        c.set_graphs(True)
        c.eom_sigma("ea", x)
        out.append((c.eom_sigma("ea", x), plain))
    for got, plain in out:
        assert np.array_equal(got, plain)
    assert not np.array_equal(out[0][0], out[1][0])
    c.close()


def test_solve_with_and_without_replay(pkg):
    h, eri = synth.hamiltonian(6, 10, seed=0)
    roots = []
    for graphs in (False, True):
        c = pkg.Context(0)
        c.set_graphs(graphs)
        c.fno_truncate(h, eri, 3, 1e-4)
        assert c.ccsdt_solve()["converged"]
        r = c.eom_solve("dip", 3)
        assert r["converged"]
        roots.append(r["omegas"])
        c.close()
    assert np.max(np.abs(roots[0] - roots[1])) < 1e-12


@pytest.mark.parametrize("variant", ["ip", "dea"])
def test_side_streams_match_serial(ctx, variant):
    """The component blocks of a product run on several streams (nine
    blocks into their own accumulators for IP, three output components for
    DEA); with per-launch profiling they run one after another on the
    context stream with the same accumulators and sums. Both orders give the
    same bits."""
    o, v, _ = ctx.dims()
    ctx.set_precision("fp64")
    ctx.set_graphs(False)
    x = vector(variant, o, v, 740)
    ctx.eom_sigma(variant, x)
    forked = ctx.eom_sigma(variant, x)
    ctx.profile(True)
    serial = ctx.eom_sigma(variant, x)
    ctx.profile(False)
    ctx.set_graphs(True)
    assert np.array_equal(forked, serial)
