"""The oracle's pins catch plausible mistakes (CPU, no GPU).

Each case plants one mistake in a copy of the oracle's arithmetic - a
dropped term, a flipped sign, integrals read in the wrong index order, a
wrong evaluation point, a wrong-signed gradient block, a dropped factor -
and checks that the independent reference the pins use (the Fock-space
definition, the closed form on linear data, finite differences, second-order
perturbation theory in determinant space) no longer agrees. A pin that still passed here would not protect the
oracle against that mistake.
"""
import math

import numpy as np
import pytest

import synth
from oracle import detspace, fno, packing, wick, xfno


@pytest.fixture(scope="module")
def small():
    nocc, n = 2, 5
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 21)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    amps = {}
    for r in (1, 2, 3):
        x = synth.random_packed(math.comb(o, r) * math.comb(v, r), 40 + r, 0.1)
        amps[r] = packing.unpack(x * synth.packed_ms_mask(r, r, o, v, 0), r, r, o, v)
    return ham, amps, detspace.DefinitionOracle(ham["hso"], ham["g"], o)


def _largest_term(terms, nh, np_, ham, a, o, v):
    sizes = [np.max(np.abs(wick.evaluate((t,), nh, np_, ham["f"], ham["g"], a, o, v))) for t in terms]
    return int(np.argmax(sizes))


@pytest.mark.parametrize("mistake", ["drop", "sign"])
def test_cc_definition_pin_catches_a_bad_term(small, mistake):
    ham, amps, dso = small
    o, v = ham["o"], ham["v"]
    a = {"t1": amps[1], "t2": amps[2], "t3": amps[3]}
    terms = list(wick.cc_terms(3))
    k = _largest_term(terms, 3, 3, ham, a, o, v)
    if mistake == "drop":
        del terms[k]
    else:
        terms[k] = (terms[k][0], -terms[k][1])
    got = wick.evaluate(tuple(terms), 3, 3, ham["f"], ham["g"], a, o, v)
    ref = dso.cc_residual(amps, 3)
    assert np.max(np.abs(got - ref)) > 1e-6


def test_eom_definition_pin_catches_a_misordered_integral(small):
    ham, amps, dso = small
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES["ip"]
    rs = [packing.unpack(synth.random_packed(packing.packed_size(nh, np_, o, v), 90 + k, 0.3), nh, np_, o, v)
          for k, (nh, np_) in enumerate(comps)]
    a = {"t1": amps[1], "t2": amps[2], "t3": amps[3], "r1": rs[0], "r2": rs[1], "r3": rs[2]}
    terms = wick.eom_terms("ip", 1, 1)
    # <pq||rs> read in chemists' order (<pr||qs>): the index-order mistake
    gbad = ham["g"].transpose(0, 2, 1, 3)
    got = wick.evaluate(terms, 2, 1, ham["f"], gbad, a, o, v)
    ref = dso.eom_sigma(amps, [(rs[k],) + comps[k] for k in range(3)], 2, 1) - sum(
        wick.evaluate(wick.eom_terms("ip", 1, ic), 2, 1, ham["f"], ham["g"], a, o, v) for ic in (0, 2))
    good = wick.evaluate(terms, 2, 1, ham["f"], ham["g"], a, o, v)
    assert np.max(np.abs(good - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(got - ref)) > 1e-6


def test_xfno_pin_catches_the_wrong_evaluation_point():
    f = np.array([0.999, 0.9975, 0.995])
    e = -1.2 + 0.4 * (1 - f)          # linear data: the extrapolation must return -1.2
    assert abs(xfno.extrapolate(f, e) + 1.2) < 1e-12
    slope, icpt = np.polyfit(f, e, 1)
    assert abs(icpt + 1.2) > 1e-3      # evaluating at f = 0 instead of 1 would fail the pin


def test_mlp_gradient_pin_catches_a_wrong_layer_gradient():
    """The finite-difference pin of the guess network's gradient rejects a
    gradient whose hidden-layer bias block has the wrong sign."""
    from oracle import mlp
    rng = np.random.default_rng(3)
    width, n = 5, 7
    nparam = mlp.NIN * width + width + width * width + width + width * mlp.NOUT + mlp.NOUT
    params = rng.normal(0, 0.5, nparam)
    x, t = rng.normal(0, 1.0, (n, mlp.NIN)), rng.normal(0, 1.0, (n, mlp.NOUT))
    w = rng.uniform(0.2, 1.5, (n, mlp.NOUT))
    _, g = mlp.loss_grad(params, x, t, w, width)
    bad = g.copy()
    b1 = slice(mlp.NIN * width, mlp.NIN * width + width)   # first bias block (parameter layout)
    bad[b1] = -bad[b1]
    h = 1e-6
    fd = np.array([(mlp.loss_grad(params + h * e, x, t, w, width)[0]
                    - mlp.loss_grad(params - h * e, x, t, w, width)[0]) / (2 * h) for e in np.eye(nparam)])
    tol = 1e-7 * max(1.0, np.max(np.abs(fd)))
    assert np.max(np.abs(g - fd)) < tol
    assert np.max(np.abs(bad - fd)) > tol


def test_mp2_density_pin_catches_a_dropped_half():
    """Second-order perturbation theory in determinant space rejects the
    vv density without the 1/2 of Eq. 10."""
    h, eri = synth.hamiltonian(4, 5, seed=2)
    scf = fno.rhf(h, eri, 2)
    act = fno.active_hamiltonian(h, eri, scf["c"], 2)
    hso, g, o = act["hso"], act["g"], act["o"]
    d = fno.mp2_vv_density(act["f"], g, o)
    fs = detspace.FockSpace(hso.shape[0])
    hmat = fs.hamiltonian(hso, g)
    ref = fs.vacuum(range(o))
    eso = np.repeat(scf["eps"], 2)
    occ_energy = np.array([eso[[p for p in range(len(eso)) if (s >> p) & 1]].sum() for s in fs.states])
    hv = hmat @ ref
    e0 = occ_energy[int(np.argmax(ref))]
    n_e = np.bitwise_count(fs.states)
    psi1 = np.zeros(fs.dim)
    sel = (n_e == o) & (ref == 0) & (np.abs(hv) > 0)
    psi1[sel] = -hv[sel] / (occ_energy[sel] - e0)
    vir = list(range(o, hso.shape[0]))
    dd = np.array([[psi1 @ (fs.string([(a, True), (b, False)]) @ psi1) for b in vir] for a in vir])
    tol = 1e-10 * np.max(np.abs(d))
    assert np.max(np.abs(dd - d)) < tol
    assert np.max(np.abs(dd - 2 * d)) > tol


def test_sampled_evaluation_pin_catches_a_transposed_gather(small):
    """The sampled-element checker of the large parity cases, with its two
    hole columns swapped (a transposed external gather), no longer matches
    the Fock-space definition, while the correct gather does."""
    ham, amps, dso = small
    o, v = ham["o"], ham["v"]
    a = {"t1": amps[1], "t2": amps[2], "t3": amps[3]}
    ref = dso.cc_residual(amps, 2)
    rng = np.random.default_rng(8)
    tup = np.concatenate([rng.integers(0, o, (200, 2)), rng.integers(0, v, (200, 2))], axis=1)
    good = wick.evaluate_at(wick.cc_terms(2), 2, 2, ham["f"], ham["g"], a, o, v, tup)
    bad = wick.evaluate_at(wick.cc_terms(2), 2, 2, ham["f"], ham["g"], a, o, v, tup[:, [1, 0, 2, 3]])
    want = ref[tuple(tup.T)]
    tol = 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(good - want)) < tol
    assert np.max(np.abs(bad - want)) > 1e-6
