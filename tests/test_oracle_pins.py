"""Pins of the CPU oracle against quantities fixed by the paper's definitions
and by mathematics, independent of the oracle's own formulas.

  * CC residuals (Eq. 6) and energy (Eq. 7), and the EOM products of Eq. 1-4,
    against the Fock-space definition on random amplitudes (oracle/detspace.py);
  * CCSDT = FCI for three electrons; EOM-CCSDT = FCI for every root where
    the operator space spans the whole (N +- m) sector (IP, EA, DEA from two
    electrons, DIP from four; EE from two, its excited states);
  * MP2 energy and virtual-virtual density (Eq. 8-10) against second-order
    perturbation theory written out in determinant space;
  * RHF stationarity; invariance of CCSDT under the FNO rotation at
    threshold 0; size-extensivity; the non-interacting (Koopmans) limit;
  * XFNO exactness on linear data; truncation rules.
"""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import cc, detspace, eom, fno, mlp, packing, wick, xfno


def spin_masked(nh, np_, o, v, seed, scale, ms2=0):
    x = synth.random_packed(math.comb(o, nh) * math.comb(v, np_), seed, scale)
    return x * synth.packed_ms_mask(nh, np_, o, v, ms2)


@pytest.fixture(scope="module")
def small_system():
    nocc, n = 2, 5
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 21)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    amps = {r: packing.unpack(spin_masked(r, r, o, v, 40 + r, 0.1), r, r, o, v) for r in (1, 2, 3)}
    dso = detspace.DefinitionOracle(ham["hso"], ham["g"], o)
    return ham, amps, dso


def test_packing_roundtrip_and_signs():
    o, v = 5, 6
    for nh, np_ in [(1, 0), (0, 2), (2, 2), (3, 2), (2, 4), (4, 2)]:
        x = np.random.default_rng(nh * 10 + np_).normal(size=packing.packed_size(nh, np_, o, v))
        d = packing.unpack(x, nh, np_, o, v)
        assert np.array_equal(packing.pack(d, nh, np_, o, v), x)
        if nh >= 2:  # antisymmetric under a hole swap, zero on repeated holes
            assert np.allclose(d, -np.swapaxes(d, 0, 1))
            assert np.all(d[0, 0] == 0)
        if np_ >= 2:
            assert np.allclose(d, -np.swapaxes(d, nh, nh + 1))


@pytest.mark.parametrize("rank", [1, 2, 3])
def test_cc_residual_equals_definition(small_system, rank):
    ham, amps, dso = small_system
    o, v = ham["o"], ham["v"]
    a = {"t1": amps[1], "t2": amps[2], "t3": amps[3]}
    got = wick.evaluate(wick.cc_terms(rank), rank, rank, ham["f"], ham["g"], a, o, v)
    ref = dso.cc_residual(amps, rank)
    assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_cc_energy_equals_definition(small_system):
    ham, amps, dso = small_system
    o, v = ham["o"], ham["v"]
    e = cc.energy(ham["f"], ham["g"], o, v, amps[1], amps[2], amps[3])
    assert abs(e - dso.cc_energy(amps, ham["e_ref"])) < 1e-12


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_eom_sigma_equals_definition(small_system, variant):
    ham, amps, dso = small_system
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES[variant]
    rs = [packing.unpack(synth.random_packed(packing.packed_size(nh, np_, o, v), 90 + k, 0.3), nh, np_, o, v)
          for k, (nh, np_) in enumerate(comps)]
    got = eom.sigma_dense(variant, ham["f"], ham["g"], o, v, amps[1], amps[2], amps[3], rs)
    for oc, (nh, np_) in enumerate(comps):
        ref = dso.eom_sigma(amps, [(rs[k],) + comps[k] for k in range(3)], nh, np_)
        assert np.max(np.abs(got[oc] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), (variant, oc)


def _so_hamiltonian(h, eri):
    g = fno.spin_orbital_integrals(eri)
    hso = fno.spin_orbital_one_body(h)
    return hso, g


def test_ccsdt_three_electrons_is_fci():
    # open-shell 3-electron reference (0a, 0b, 1a) in 5 spatial orbitals
    h, eri = synth.random_symmetric_mo_hamiltonian(5, 3, scale_h=0.1, scale_eri=0.03)
    hso, g = _so_hamiltonian(h, eri)
    o = 3
    f, e_ref = fno.fock_from_bare(hso, g, o)
    res = cc.ccsdt(f, g, o, hso.shape[0] - o)
    assert res["converged"]
    e_fci = detspace.fci_energies(hso, g, 3, 1)
    assert abs(e_ref + res["e_corr"] - e_fci[0]) < 1e-9


def _dense_roots(variant, act, res, k, principal_only=False):
    """Lowest k eigenvalues (total energies) of the dense sector matrix; with
    principal_only, among eigenvectors with principal-block weight >= 1e-6."""
    f, g, o, v = act["f"], act["g"], act["o"], act["v"]
    m = eom.sigma_matrix(variant, f, g, o, v, res["t1"], res["t2"], res["t3"])
    w, vecs = np.linalg.eig(m)
    if principal_only:
        idx = np.where(eom.ms_mask(variant, o, v))[0]
        npr = int(np.sum(idx < eom.sizes(variant, o, v)[0]))
        weight = np.sum(np.abs(vecs[:npr]) ** 2, axis=0) / np.sum(np.abs(vecs) ** 2, axis=0)
        w = w[weight >= 1e-6]
    w = np.sort(w.real)
    return act["e_ref"] + res["e_corr"] + w[:k], m.shape[0]


@pytest.fixture(scope="module")
def two_electron():
    h, eri = synth.hamiltonian(2, 5, seed=36)
    act = fno.fno_truncate(h, eri, 1, 0.0)
    res = cc.ccsdt(act["f"], act["g"], act["o"], act["v"])
    return act, res


def test_ccsdt_two_electrons_is_fci(two_electron):
    act, res = two_electron
    assert res["converged"]
    e_fci = detspace.fci_energies(act["hso"], act["g"], 2, 0)
    assert abs(act["e_ref"] + res["e_corr"] - e_fci[0]) < 1e-9


@pytest.mark.parametrize("variant,nelec,ms2", [("ip", 1, 1), ("ea", 3, 1), ("dea", 4, 0)])
def test_eom_two_electron_reference_is_fci(two_electron, variant, nelec, ms2):
    act, res = two_electron
    fci = detspace.fci_energies(act["hso"], act["g"], nelec, ms2)
    roots, dim = _dense_roots(variant, act, res, len(fci))
    assert dim == len(fci)  # the operator space spans the whole sector
    assert np.max(np.abs(roots - fci)) < 1e-8


def test_ee_two_electron_reference_is_fci(two_electron):
    """EE from a two-electron reference: 1h1p and 2h2p span every other
    determinant of the N = 2, M_s = 0 sector, so E_CC + omega are the excited
    FCI energies (the ground state is the reference's own root)."""
    act, res = two_electron
    fci = detspace.fci_energies(act["hso"], act["g"], 2, 0)
    roots, dim = _dense_roots("ee", act, res, len(fci) - 1)
    assert dim == len(fci) - 1
    assert np.max(np.abs(roots - fci[1:])) < 1e-8


def _three_electron_reference():
    h, eri = synth.random_symmetric_mo_hamiltonian(4, 3, scale_h=0.1, scale_eri=0.03)
    hso, g = _so_hamiltonian(h, eri)
    o = 3
    f, e_ref = fno.fock_from_bare(hso, g, o)
    v = hso.shape[0] - o
    res = cc.ccsdt(f, g, o, v)
    assert res["converged"] and np.max(np.abs(res["t3"])) > 1e-8
    return hso, g, f, e_ref, o, v, res


def _whole_space_roots(variant, f, g, o, v, res):
    dim = sum(eom.sizes(variant, o, v))
    cols = []
    for k in range(dim):
        e = np.zeros(dim)
        e[k] = 1.0
        cols.append(eom.sigma_packed(variant, f, g, o, v, res["t1"], res["t2"], res["t3"], e))
    return np.sort(np.linalg.eigvals(np.array(cols).T).real), dim


def test_ip_three_electron_reference_is_fci():
    """IP from the open-shell three-electron reference: 1h, 2h1p and 3h2p of
    every spin change span all two-electron determinants, with T3 active,
    so E_CC + omega are all FCI energies of N = 2."""
    hso, g, f, e_ref, o, v, res = _three_electron_reference()
    w, dim = _whole_space_roots("ip", f, g, o, v, res)
    fci = np.sort(np.concatenate([detspace.fci_energies(hso, g, 2, ms2) for ms2 in (-2, 0, 2)]))
    assert dim == len(fci)
    assert np.max(np.abs(e_ref + res["e_corr"] + w - fci)) < 1e-8


def test_ee_three_electron_reference_is_fci():
    """EE from an open-shell three-electron reference (0a, 0b, 1a) in 4
    spatial orbitals: 1h1p, 2h2p and 3h3p of every spin change span every
    other three-electron determinant, CCSDT is exact and T3 is active, so
    E_CC + omega over the whole operator space are all FCI energies of N = 3
    except the ground state (the sector masks assume an even number of
    occupied spin orbitals, so the space is taken whole here)."""
    hso, g, f, e_ref, o, v, res = _three_electron_reference()
    w, dim = _whole_space_roots("ee", f, g, o, v, res)
    roots = e_ref + res["e_corr"] + w
    fci = np.sort(np.concatenate([detspace.fci_energies(hso, g, 3, ms2) for ms2 in (-3, -1, 1, 3)]))
    assert dim == len(fci) - 1
    ground = int(np.argmin(np.abs(fci - (e_ref + res["e_corr"]))))
    assert abs(fci[ground] - (e_ref + res["e_corr"])) < 1e-9
    assert np.max(np.abs(roots - np.delete(fci, ground))) < 1e-8


def test_dip_four_electron_reference_is_fci():
    h, eri = synth.hamiltonian(4, 5, seed=2)
    act = fno.fno_truncate(h, eri, 2, 0.0)
    res = cc.ccsdt(act["f"], act["g"], act["o"], act["v"])
    assert res["converged"]
    assert np.max(np.abs(res["t3"])) > 1e-6  # triples are active here
    fci = detspace.fci_energies(act["hso"], act["g"], 2, 0)
    roots, dim = _dense_roots("dip", act, res, len(fci))
    assert dim == len(fci)
    assert np.max(np.abs(roots - fci)) < 1e-8


def test_left_product_is_the_transposed_product(two_electron):
    """The left product is L times the product matrix: its dense matrix is
    the transpose of the right one, the left eigenvalues equal the right
    ones, and left and right eigenvectors of distinct roots are
    biorthogonal."""
    act, res = two_electron
    f, g, o, v = act["f"], act["g"], act["o"], act["v"]
    variant = "ip"
    mask = eom.ms_mask(variant, o, v)
    idx = np.where(mask)[0]
    m = eom.sigma_matrix(variant, f, g, o, v, res["t1"], res["t2"], res["t3"])
    rng = np.random.default_rng(5)
    lvec = np.zeros(len(mask))
    lvec[idx] = rng.normal(size=len(idx))
    lam = eom.left_sigma_packed(variant, f, g, o, v, res["t1"], res["t2"], res["t3"], lvec)
    assert np.max(np.abs(lam[idx] - m.T @ lvec[idx])) < 1e-12
    assert np.all(lam[~mask] == 0)
    wr, vr = np.linalg.eig(m)
    wl, vl = np.linalg.eig(m.T)
    assert np.max(np.abs(np.sort(wr.real) - np.sort(wl.real))) < 1e-10
    order_r, order_l = np.argsort(wr.real), np.argsort(wl.real)
    overlap = vl[:, order_l].T @ vr[:, order_r]
    off = overlap - np.diag(np.diag(overlap))
    gaps = np.min(np.abs(np.subtract.outer(wr.real, wr.real)) + np.eye(len(wr)) * 1e9)
    assert gaps > 1e-8 and np.max(np.abs(off)) < 1e-8


def test_davidson_matches_dense_diagonalisation():
    h, eri = synth.hamiltonian(4, 5, seed=2)
    act = fno.fno_truncate(h, eri, 2, 0.0)
    f, g, o, v = act["f"], act["g"], act["o"], act["v"]
    res = cc.ccsdt(f, g, o, v)
    for variant in ("ip", "dea"):
        dense, _ = _dense_roots(variant, act, res, 3, principal_only=True)
        out = eom.eom_ccsdt(variant, f, g, o, v, res["t1"], res["t2"], res["t3"], 3, tol_res=1e-9)
        assert out["converged"]
        got = act["e_ref"] + res["e_corr"] + out["omega"]
        assert np.max(np.abs(got - dense)) < 1e-9, (variant, got, dense)


def test_davidson_returns_lowest_principal_states():
    """Six electrons in five orbitals: the IP operator space holds quartet
    2h1p states with no 1h weight below the third doublet root (and DIP
    quintet 3h1p states likewise). The roots are the lowest eigenvalues of
    the dense sector matrix among eigenvectors with principal-block weight
    (at least 1e-6); the zero-weight states are excluded, not missed."""
    h, eri = synth.hamiltonian(6, 5, seed=0)
    act = fno.fno_truncate(h, eri, 3, 0.0)
    f, g, o, v = act["f"], act["g"], act["o"], act["v"]
    res = cc.ccsdt(f, g, o, v)
    assert res["converged"]
    variant = "ip"
    m = eom.sigma_matrix(variant, f, g, o, v, res["t1"], res["t2"], res["t3"])
    w, vecs = np.linalg.eig(m)
    idx = np.where(eom.ms_mask(variant, o, v))[0]
    npr = int(np.sum(idx < eom.sizes(variant, o, v)[0]))
    weight = np.sum(np.abs(vecs[:npr]) ** 2, axis=0) / np.sum(np.abs(vecs) ** 2, axis=0)
    order = np.argsort(w.real)
    principal = [w[j].real for j in order if weight[j] >= 1e-6][:3]
    # the pin means something: a zero-weight state lies below the third root
    assert any(weight[j] < 1e-12 and w[j].real < principal[-1] for j in order)
    out = eom.eom_ccsdt(variant, f, g, o, v, res["t1"], res["t2"], res["t3"], 3, tol_res=1e-9)
    assert out["converged"]
    assert np.max(np.abs(out["omega"] - np.array(principal))) < 1e-9, (out["omega"], principal)


def test_mp2_energy_and_density_from_perturbation_theory():
    h, eri = synth.hamiltonian(4, 5, seed=2)
    scf = fno.rhf(h, eri, 2)
    c, eps = scf["c"], scf["eps"]
    act = fno.active_hamiltonian(h, eri, c, 2)
    hso, g, o = act["hso"], act["g"], act["o"]
    # oracle formulas (Eq. 8-10)
    t2 = fno.mp2_amplitudes(act["f"], g, o)
    e2 = fno.mp2_energy(g, t2, o)
    d = fno.mp2_vv_density(act["f"], g, o)
    # determinant space: |psi1> = -sum_D |D><D|H|0> / (E_D - E_0), H0 = sum eps_p n_p
    fs = detspace.FockSpace(hso.shape[0])
    hmat = fs.hamiltonian(hso, g)
    ref = fs.vacuum(range(o))
    eso = np.repeat(eps, 2)
    occ_energy = np.array([eso[[p for p in range(len(eso)) if (s >> p) & 1]].sum() for s in fs.states])
    hv = hmat @ ref
    e0 = occ_energy[int(np.argmax(ref))]
    n_e = np.bitwise_count(fs.states)
    psi1 = np.zeros(fs.dim)
    sel = (n_e == o) & (ref == 0) & (np.abs(hv) > 0)
    psi1[sel] = -hv[sel] / (occ_energy[sel] - e0)
    assert abs(ref @ hmat @ psi1 - e2) < 1e-12
    vir = list(range(o, hso.shape[0]))
    dd = np.array([[psi1 @ (fs.string([(a, True), (b, False)]) @ psi1) for b in vir] for a in vir])
    assert np.max(np.abs(dd - d)) < 1e-10 * np.max(np.abs(d))


def test_rhf_is_stationary_and_matches_determinant_energy():
    h, eri = synth.hamiltonian(6, 10, seed=0)
    scf = fno.rhf(h, eri, 3)
    act = fno.active_hamiltonian(h, eri, scf["c"], 3)
    o = act["o"]
    assert np.max(np.abs(act["f"][:o, o:])) < 1e-9               # Brillouin
    assert abs(act["e_ref"] - scf["e"]) < 1e-10                    # <Phi0|H|Phi0>
    assert np.max(np.abs(np.diag(act["f"]) - np.repeat(scf["eps"], 2))) < 1e-9
    assert np.max(np.abs(scf["d"] @ scf["d"] - scf["d"])) < 1e-12  # idempotent


def test_threshold_zero_reproduces_untruncated_ccsdt():
    h, eri = synth.hamiltonian(4, 6, seed=0)
    trunc = fno.fno_truncate(h, eri, 2, 0.0)
    assert trunc["nkept"] == 4 and abs(trunc["kept_fraction"] - 1.0) < 1e-15
    scf = fno.rhf(h, eri, 2)
    canon = fno.active_hamiltonian(h, eri, scf["c"], 2)
    e1 = cc.ccsdt(trunc["f"], trunc["g"], trunc["o"], trunc["v"])["e_corr"]
    e2 = cc.ccsdt(canon["f"], canon["g"], canon["o"], canon["v"])["e_corr"]
    assert abs(e1 - e2) < 1e-10


def test_size_extensivity_of_ccsdt():
    ha, ea = synth.random_symmetric_mo_hamiltonian(3, 5, scale_h=0.1, scale_eri=0.05)
    hb, eb = synth.random_symmetric_mo_hamiltonian(3, 6, scale_h=0.1, scale_eri=0.05)
    # well-separated occupied / virtual levels so that each fragment has a clear reference
    ha[np.diag_indices(3)] = [-1.1, 0.6, 1.4]
    hb[np.diag_indices(3)] = [-0.9, 0.8, 1.2]
    # combined orbital order: occupied A, occupied B, virtuals A, virtuals B
    order = [("a", 0), ("b", 0), ("a", 1), ("a", 2), ("b", 1), ("b", 2)]
    n = len(order)
    h = np.zeros((n, n))
    eri = np.zeros((n,) * 4)
    for p, (sp, ip) in enumerate(order):
        for q, (sq, iq) in enumerate(order):
            if sp == sq:
                h[p, q] = (ha if sp == "a" else hb)[ip, iq]
    for idx in itertools.product(range(n), repeat=4):
        sys_ = {order[k][0] for k in idx}
        if len(sys_) == 1:
            src = ea if "a" in sys_ else eb
            eri[idx] = src[tuple(order[k][1] for k in idx)]
    e = {}
    for name, (hh, ee, nocc) in {"a": (ha, ea, 1), "b": (hb, eb, 1), "ab": (h, eri, 2)}.items():
        ham = fno.mo_hamiltonian(hh, ee, nocc)
        res = cc.ccsdt(ham["f"], ham["g"], ham["o"], ham["v"], tol_res=1e-12, tol_e=1e-14)
        assert res["converged"]
        e[name] = res["e_corr"]
    assert abs(e["ab"] - e["a"] - e["b"]) < 1e-10


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_noninteracting_limit_is_koopmans(variant):
    n, nocc = 5, 2
    eps = np.array([-1.3, -0.7, 0.4, 0.9, 1.6])
    ham = fno.mo_hamiltonian(np.diag(eps), np.zeros((n,) * 4), nocc)
    f, g, o, v = ham["f"], ham["g"], ham["o"], ham["v"]
    res = cc.ccsdt(f, g, o, v)
    assert abs(res["e_corr"]) < 1e-14
    out = eom.eom_ccsdt(variant, f, g, o, v, res["t1"], res["t2"], res["t3"], 3)
    eso = np.repeat(eps, 2)
    occ, vir = list(range(o)), list(range(o, 2 * n))
    spin = lambda p: 1 if p % 2 == 0 else -1
    # eigenvectors are single determinants here: the roots are the lowest
    # principal-block (1h / 1p / 2h / 2p) determinant energies of the sector
    # (the others carry no principal weight), filled up by the lowest others
    # where the sector has fewer than three principal determinants
    vals = [[], []]
    for k, (nh, np_) in enumerate(wick.EOM_SPACES[variant]):
        for hs in itertools.combinations(occ, nh):
            for ps in itertools.combinations(vir, np_):
                if sum(spin(a) for a in ps) - sum(spin(i) for i in hs) == eom.SECTOR_MS2[variant]:
                    vals[min(k, 1)].append(sum(eso[a] for a in ps) - sum(eso[i] for i in hs))
    principal = sorted(vals[0])[:3]
    expect = np.sort(principal + sorted(vals[1])[:3 - len(principal)])
    assert np.max(np.abs(np.sort(out["omega"]) - expect)) < 1e-10


def test_xfno_is_exact_on_linear_data():
    f = np.array([0.999, 0.9975, 0.995])
    e = -1.5 + 0.3 * (1 - f)
    assert abs(xfno.extrapolate(f, e) + 1.5) < 1e-14
    assert abs(xfno.extrapolate([1.0, 1.0], [-2.0, -2.0]) + 2.0) < 1e-15


def test_truncation_rules():
    occ = np.array([1e-2, 5e-3, 1e-4, 1e-4, 5e-5, 1e-6])
    assert fno.choose_kept(occ, 1e-4) == 4
    assert fno.choose_kept(occ, 0.0) == 6
    assert fno.choose_kept(occ, 1.0) == 0
    assert fno.choose_kept(occ, 0.5, nkeep=2) == 2
    tot = occ.sum()
    assert fno.choose_kept(occ, (occ[0] + occ[1]) / tot, criterion="occt") == 2
    # a degenerate pair straddling the cut is kept whole
    occ2 = np.array([1e-2, 2e-3, 2e-3, 1e-5])
    assert fno.choose_kept(occ2, (occ2[0] + occ2[1]) / occ2.sum(), criterion="occt") == 3


# ---- learned-guess network (oracle/mlp.py) -----------------------------------------

def _mlp_case(width=5, n=7, seed=3):
    rng = np.random.default_rng(seed)
    nparam = mlp.NIN * width + width + width * width + width + width * mlp.NOUT + mlp.NOUT
    params = rng.normal(0, 0.5, nparam)
    x = rng.normal(0, 1.0, (n, mlp.NIN))
    t = rng.normal(0, 1.0, (n, mlp.NOUT))
    w = rng.uniform(0.2, 1.5, (n, mlp.NOUT))
    return params, x, t, w, width


def test_mlp_gradient_matches_finite_differences():
    params, x, t, w, width = _mlp_case()
    _, g = mlp.loss_grad(params, x, t, w, width)
    h = 1e-6
    fd = np.zeros_like(params)
    for i in range(params.size):
        e = np.zeros_like(params)
        e[i] = h
        fd[i] = (mlp.loss_grad(params + e, x, t, w, width)[0] - mlp.loss_grad(params - e, x, t, w, width)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_mlp_zero_weights_closed_form():
    params, x, t, w, width = _mlp_case()
    layers = mlp.unpack(params, width)
    b3 = np.array([0.3, -1.2])
    zero = mlp.pack([np.zeros_like(layers[0]), layers[1], np.zeros_like(layers[2]), layers[3],
                     np.zeros_like(layers[4]), b3])
    y, _ = mlp.forward(zero, x, width)
    assert np.allclose(y, b3)  # no path from the input: the output bias alone
    loss, g = mlp.loss_grad(zero, x, t, w, width)
    assert abs(loss - np.sum(w * (b3 - t) ** 2) / len(x)) < 1e-14
    gl = mlp.unpack(g, width)
    assert np.allclose(gl[5], np.sum(2 * w * (b3 - t), axis=0) / len(x))
    assert np.all(gl[0] == 0) and np.all(gl[2] == 0)  # zero weights above pass nothing back


def test_adam_first_step_is_signed_learning_rate():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first moments equal g and g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(new, p - 0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_eom_features_definition():
    # 2 occupied / 4 virtual spin orbitals (alpha even), IP spaces (1h, 2h1p,
    # 3h2p); integrals <0 3||0 3> = 0.25 (alpha hole 0, beta particle 1) and
    # <0 2||0 2> = 0.1 (same spin, other spatial orbital pair entry)
    o, v = 2, 4
    fdiag = np.array([-1.0, -0.8, 0.5, 0.7, 1.1, 1.3])
    g = np.zeros((6,) * 4)
    for p, q, val in [(0, 3, 0.25), (0, 2, 0.1)]:
        for a, b in [(p, q), (q, p)]:
            g[a, b, a, b] = val
            g[a, b, b, a] = -val
    occ = np.array([1e-2, 1e-4])
    feats = mlp.eom_features(wick.EOM_SPACES["ip"], 0, fdiag, g, o, v, occ)
    assert feats.shape == (2 + 1 * 4 + 0, 8)  # C(2,3) = 0: no 3h2p element
    assert np.allclose(feats[0], [1.0, 0.0, -1.0, 0.0, 0.0, 0.0, 0, 0])
    # holes 0,1 and particle 1 (orbital 3): the hole 0 - particle pair lowers
    # the energy by the spin average of <03||03> and <02||02>
    assert np.allclose(feats[2 + 1], [0.7 + 1.8, -0.5 * (0.25 + 0.1), -0.8, 0.7, 0.7, -2.0, 1, 0])
    # particle 0 (orbital 2, same spatial orbital as 3): the same average
    assert np.allclose(feats[2 + 0], [0.5 + 1.8, -0.5 * (0.1 + 0.25), -0.8, 0.5, 0.5, -2.0, 1, 0])
    # holes 0,1 and particle 2 (orbital 4, virtual spatial 1): no integral
    assert np.allclose(feats[2 + 2], [1.1 + 1.8, 0.0, -0.8, 1.1, 1.1, -4.0, 1, 0])


def test_en_shift_from_spatial_coulomb_and_exchange():
    """The spin-averaged two-body shift against J and K built directly from
    the spatial chemists' integrals (an independent route): for every element
    of a small DIP space, sum over pairs of +-(J_PP or J_PQ - K_PQ/2); and all
    features are equal for an element and its spin-flipped partner."""
    h, eri = synth.random_symmetric_mo_hamiltonian(4, 17)
    ham = fno.mo_hamiltonian(h, eri, 2)
    o, v = ham["o"], ham["v"]
    feats = mlp.eom_features(wick.EOM_SPACES["dip"], 2, np.diag(ham["f"]), ham["g"], o, v)
    jmat = np.einsum("ppqq->pq", eri)
    kmat = np.einsum("pqqp->pq", eri)
    rows = {}
    row = 0
    for comp, (nh, np_) in enumerate(wick.EOM_SPACES["dip"]):
        for hs in itertools.combinations(range(o), nh):
            for ps in itertools.combinations(range(v), np_):
                orbs = list(hs) + [o + a for a in ps]
                en = 0.0
                for x in range(len(orbs)):
                    for y in range(x + 1, len(orbs)):
                        sp, sq = orbs[x] // 2, orbs[y] // 2
                        w = jmat[sp, sp] if sp == sq else jmat[sp, sq] - 0.5 * kmat[sp, sq]
                        en += w if (x < nh) == (y < nh) else -w
                assert abs(feats[row, 1] - en) < 1e-12
                rows[(comp, hs, ps)] = row
                row += 1
    assert row == feats.shape[0]
    for (comp, hs, ps), r in rows.items():
        fh = tuple(sorted(i ^ 1 for i in hs))
        fp = tuple(sorted(a ^ 1 for a in ps))
        assert np.allclose(feats[r], feats[rows[(comp, fh, fp)]])


def _random_tuples(o, v, nh, np_, count, seed):
    """Output elements in any index order (unsorted, repeated indices
    included), so that a transposed gather in the sampled evaluation shows."""
    rng = np.random.default_rng(seed)
    hs = rng.integers(0, o, size=(count, nh))
    ps = rng.integers(0, v, size=(count, np_))
    return np.concatenate([hs, ps], axis=1)


@pytest.mark.parametrize("rank", [1, 2, 3])
def test_sampled_cc_residual_equals_definition(small_system, rank):
    """wick.evaluate_at (the checker of the large parity cases) against the
    Fock-space definition at arbitrary output elements."""
    ham, amps, dso = small_system
    o, v = ham["o"], ham["v"]
    a = {"t1": amps[1], "t2": amps[2], "t3": amps[3]}
    ref = dso.cc_residual(amps, rank)
    tup = _random_tuples(o, v, rank, rank, 400, 60 + rank)
    got = wick.evaluate_at(wick.cc_terms(rank), rank, rank, ham["f"], ham["g"], a, o, v, tup)
    want = ref[tuple(tup.T)]
    assert np.max(np.abs(got - want)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea", "ee"])
def test_sampled_eom_sigma_equals_definition(small_system, variant):
    ham, amps, dso = small_system
    o, v = ham["o"], ham["v"]
    comps = wick.EOM_SPACES[variant]
    rs = [packing.unpack(synth.random_packed(packing.packed_size(nh, np_, o, v), 95 + k, 0.3), nh, np_, o, v)
          for k, (nh, np_) in enumerate(comps)]
    a = {"t1": amps[1], "t2": amps[2], "t3": amps[3], "r1": rs[0], "r2": rs[1], "r3": rs[2]}
    for oc, (nh, np_) in enumerate(comps):
        ref = dso.eom_sigma(amps, [(rs[k],) + comps[k] for k in range(3)], nh, np_)
        tup = _random_tuples(o, v, nh, np_, 300, 70 + oc)
        got = sum(wick.evaluate_at(wick.eom_terms(variant, oc, ic), nh, np_, ham["f"], ham["g"], a, o, v, tup)
                  for ic in range(3))
        want = ref[tuple(tup.T)]
        assert np.max(np.abs(got - want)) < 1e-12 * max(1.0, np.max(np.abs(ref))), (variant, oc)
