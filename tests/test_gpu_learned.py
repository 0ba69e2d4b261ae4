"""Learned Davidson guess on the GPU: the network's kernels against the
oracle (oracle/mlp.py), its features and training targets against the
oracle's definitions, and solves with the learned start against plain
Davidson: the roots never depend on the network, and a trained network
saves products."""
import numpy as np
import pytest

import synth
from oracle import eom, fno, mlp, packing, wick

pytestmark = pytest.mark.gpu

WIDTH = 64


@pytest.fixture(scope="module")
def pkg():
    import paper_2509_14157_gb300 as p
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def case(n=300, seed=0):
    rng = np.random.default_rng(seed)
    nparam = mlp.NIN * WIDTH + WIDTH + WIDTH * WIDTH + WIDTH + WIDTH * mlp.NOUT + mlp.NOUT
    params = (rng.normal(0, 0.3, nparam)).astype(np.float32)
    x = rng.normal(0, 1.0, (n, mlp.NIN)).astype(np.float32)
    t = rng.normal(0, 1.0, (n, mlp.NOUT)).astype(np.float32)
    w = rng.uniform(0.2, 1.5, (n, mlp.NOUT)).astype(np.float32)
    return params, x, t, w


def test_forward_fp32_and_bf16_match_oracle(pkg):
    params, x, _, _ = case()
    net = pkg.Mlp(0, WIDTH, seed=1)
    net.set_params(params)
    ref, _ = mlp.forward(params.astype(np.float64), x.astype(np.float64), WIDTH)
    scale = np.max(np.abs(ref))
    y32 = net.forward(x)
    assert np.max(np.abs(y32 - ref)) < 1e-5 * scale
    y16 = net.forward(x, bf16=True)  # BF16 operands (8 significant bits), FP32 accumulation
    assert np.max(np.abs(y16 - ref)) < 3e-2 * scale
    net.close()


def test_loss_and_gradient_match_oracle(pkg):
    params, x, t, w = case(n=5000, seed=2)  # several row splits of the weight-gradient reduction
    net = pkg.Mlp(0, WIDTH, seed=1)
    net.set_params(params)
    loss, g = net.loss_grad(x, t, w)
    ref_loss, ref_g = mlp.loss_grad(params.astype(np.float64), x.astype(np.float64), t, w, WIDTH)
    assert abs(loss - ref_loss) < 1e-5 * abs(ref_loss)
    assert np.max(np.abs(g - ref_g)) < 1e-4 * np.max(np.abs(ref_g))
    net.close()


def test_one_training_step_is_one_adam_step(pkg):
    params, x, t, w = case(n=700, seed=3)
    net = pkg.Mlp(0, WIDTH, seed=1)
    net.set_params(params)
    hist = net.train(x, t, w, epochs=1, batch=4096, lr=1e-2)
    p64 = params.astype(np.float64)
    ref_loss, g = mlp.loss_grad(p64, x.astype(np.float64), t, w, WIDTH)
    new, _, _ = mlp.adam_step(p64, g, np.zeros_like(p64), np.zeros_like(p64), 1, lr=1e-2)
    got = net.get_params()
    # the first Adam step moves every parameter by ~lr * sign(g); elements
    # with |g| far below the FP32 rounding of g may take either sign
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(got[big] - new[big])) < 1e-5
    assert np.max(np.abs(got - new)) <= 2e-2 + 1e-6
    assert abs(hist[0] - ref_loss) < 1e-5 * abs(ref_loss)
    net.close()


def test_parameter_file_round_trip(pkg, tmp_path):
    """A trained network written to a file and read into a fresh one gives the
    same parameters and outputs; a file of another shape, a truncated file and
    a foreign file are rejected without touching the parameters."""
    params, x, t, w = case(n=700, seed=4)
    net = pkg.Mlp(0, WIDTH, seed=1)
    net.set_params(params)
    net.train(x, t, w, epochs=2, batch=256, lr=1e-3)
    path = tmp_path / "guess.bin"
    net.save(path)
    assert path.stat().st_size == 32 + 4 * net.nparam
    other = pkg.Mlp(0, WIDTH, seed=7)
    other.load(path)
    assert np.array_equal(other.get_params(), net.get_params())
    assert np.array_equal(other.forward(x[:50]), net.forward(x[:50]))
    wide = pkg.Mlp(0, 2 * WIDTH, seed=1)
    wide_before = wide.get_params()
    with pytest.raises(pkg.FnoccError):
        wide.load(path)
    assert np.array_equal(wide.get_params(), wide_before)
    cut = tmp_path / "cut.bin"
    cut.write_bytes(path.read_bytes()[:-4])
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a network" * 8)
    fresh = pkg.Mlp(0, WIDTH, seed=7)
    before = fresh.get_params()
    for bad in (cut, junk, tmp_path / "missing.bin"):
        with pytest.raises(pkg.FnoccError):
            fresh.load(bad)
        assert np.array_equal(fresh.get_params(), before)
    for m in (net, other, wide, fresh):
        m.close()


@pytest.mark.parametrize("variant", ["ip", "ea", "dip", "dea"])
def test_features_match_oracle(pkg, variant):
    h, eri = synth.hamiltonian(6, 10, seed=0)
    act = fno.fno_truncate(h, eri, 3, 1e-4)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, 3, 1e-4)
    got = ctx.eom_features(variant)
    ref = mlp.eom_features(wick.EOM_SPACES[variant], ["ip", "ea", "dip", "dea"].index(variant),
                           np.diag(act["f"]), act["g"], act["o"], act["v"], act["virt_occ"])
    assert got.shape == ref.shape
    assert np.max(np.abs(got[:, :5] - ref[:, :5])) < 1e-5 * max(1.0, np.max(np.abs(ref[:, :5])))
    assert np.max(np.abs(got[:, 5] - ref[:, 5])) < 1e-4
    assert np.array_equal(got[:, 6:], ref[:, 6:])
    ctx.close()


@pytest.mark.parametrize("variant", ["ip", "dip"])
def test_exact_diagonal_matches_oracle(pkg, variant):
    """fnocc_eom_diagonal (one product per element) against the diagonal of
    the oracle's explicit sector matrix, random amplitudes."""
    from math import comb
    nocc, n = 2, 5
    h, eri = synth.random_symmetric_mo_hamiltonian(n, 29)
    ham = fno.mo_hamiltonian(h, eri, nocc)
    o, v = ham["o"], ham["v"]
    t = [synth.random_packed(comb(o, r) * comb(v, r), 40 + r, 0.05) * synth.packed_ms_mask(r, r, o, v, 0)
         for r in (1, 2, 3)]
    ctx = pkg.Context(0)
    ctx.set_mo_hamiltonian(h, eri, nocc)
    ctx.set_amplitudes(*t)
    got = ctx.eom_diagonal(variant)
    td = [packing.unpack(t[r - 1], r, r, o, v) for r in (1, 2, 3)]
    m = eom.sigma_matrix(variant, ham["f"], ham["g"], o, v, *td)
    idx = np.where(eom.ms_mask(variant, o, v))[0]
    assert np.max(np.abs(got[idx] - np.diag(m))) < 1e-10
    assert np.all(got[np.setdiff1d(np.arange(got.size), idx)] == 0)
    # the sampled form: chosen elements, in any order, with repeats and
    # elements outside the sector (0), equal to the full diagonal there
    rng = np.random.default_rng(3)
    pick = np.concatenate([rng.choice(got.size, 12, replace=False), idx[:2], [0]])
    part = ctx.eom_diagonal(variant, pick)
    assert np.array_equal(part, got[pick])
    assert ctx.eom_diagonal(variant, np.zeros(0, dtype=np.int64)).size == 0
    for bad in ([-1], [got.size]):
        with pytest.raises(pkg.FnoccError):
            ctx.eom_diagonal(variant, bad)
    ctx.close()


def test_trained_network_saves_products_and_keeps_roots(pkg):
    """Train on small seeded systems, solve a larger held-out one: the
    learned start reaches the same roots (plain Davidson criteria) with
    fewer sigma products than the Koopmans start."""
    from paper_2509_14157_gb300 import learned
    systems = learned.seeded_training_systems(count=12)
    X, T, W, _ = learned.training_set(systems, ["dip", "dea"], 3)
    net, hist = learned.train_guess_model(X, T, W, epochs=30, batch=2048)
    assert hist[-1] < 0.5 * hist[0]
    h, eri = synth.hamiltonian(8, 20, seed=1)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, 4, 1e-4)
    assert ctx.ccsdt_solve()["converged"]
    ctx.set_guess_model(net)
    plain = with_net = 0
    for var in ("dip", "dea"):
        a = ctx.eom_solve(var, 4, guess="koopmans")
        b = ctx.eom_solve(var, 4, guess="learned")
        assert a["converged"] and b["converged"] and b["guess_used"] == 2
        assert np.max(np.abs(a["omegas"] - b["omegas"])) < 1e-9
        plain += a["sigma_calls"]
        with_net += b["sigma_calls"]
    assert with_net < plain, (with_net, plain)
    ctx.close()
    net.close()


def test_training_set_threads_and_sampled_targets(pkg):
    """The training set built on two host threads (one context each) equals
    the one built on one, with sampled exact-diagonal targets: each sampled
    correction equals the full diagonal's, the others carry weight 0."""
    from paper_2509_14157_gb300 import learned
    systems = learned.seeded_training_systems(count=4, electrons=(6, 8))
    one = learned.training_set(systems, ["ip", "dea"], 2, diag_samples=8)
    two = learned.training_set(systems, ["ip", "dea"], 2, diag_samples=8, workers=2)
    for a, b in zip(one[:3], two[:3]):
        assert np.array_equal(a, b)
    assert one[3] == two[3]
    X, T, W, info = one
    assert np.all(W[:, 0] == 1.0)  # sector elements only
    per_space = [n for _, _, n in info]
    assert np.sum(W[:, 1]) <= 8 * len(per_space) and np.sum(W[:, 1]) > 0
    full = learned.training_set(systems[:1], ["ip"], 2)
    samp = learned.training_set(systems[:1], ["ip"], 2, diag_samples=8)
    assert np.array_equal(full[0], samp[0])
    on = samp[2][:, 1] > 0
    assert np.array_equal(samp[1][on, 1], full[1][on, 1])
