"""Batched independent solves (several contexts and streams on one GPU)
against the same systems solved one by one: identical energies.

Each system runs the whole path on its own context; the kernels are
deterministic (no atomics), so concurrency must not change a single result
beyond the convergence tolerance of the solvers."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2509_14157_gb300 as p
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def small_systems():
    out = []
    # (electrons, orbitals, seed, nkeep)
    for ne, n, seed, nkeep in [(6, 10, 0, 5), (6, 10, 0, 0), (4, 9, 1, 4), (6, 11, 3, 5), (8, 12, 2, 0)]:
        h, eri = synth.hamiltonian(ne, n, seed=seed)
        out.append(dict(h=h, eri=eri, nocc=ne // 2, threshold=1e-4, nkeep=nkeep))
    return out


def solo(pkg, sy, variants, nroots):
    """The same pipeline through single calls: (status, e_ccsdt, omegas)."""
    ctx = pkg.Context(0)
    try:
        fi = ctx.fno_truncate(sy["h"], sy["eri"], sy["nocc"], sy["threshold"], nkeep=sy["nkeep"])
        if sy["nkeep"]:
            assert fi["nkept"] == sy["nkeep"]
        cc = ctx.ccsdt_solve()
        status = 0 if cc["converged"] else 1
        om = []
        for var in variants:
            r = ctx.eom_solve(var, nroots)
            status = status or (0 if r["converged"] else 1)
            om.append(r["omegas"])
        return status, cc["e_tot"], np.array(om)
    except pkg.FnoccError as err:
        return err.status, None, None
    finally:
        ctx.close()


def test_batch_equals_solo(pkg):
    systems = small_systems()
    variants = ["ip", "ea"]
    om, info = pkg.batch_solve(systems, variants, 2, nworkers=3)
    assert om.shape == (len(systems), 2, 2)
    statuses = [i["status"] for i in info]
    assert sum(st == 0 for st in statuses) >= 3, statuses
    for s, sy in enumerate(systems):
        st, e_cc, om_solo = solo(pkg, sy, variants, 2)
        assert st == statuses[s], (s, st, statuses[s])
        if st != 0:
            continue
        assert abs(e_cc - info[s]["e_ccsdt"]) < 1e-9
        assert np.max(np.abs(om_solo - om[s])) < 1e-9, s


def test_batch_rejects_bad_input(pkg):
    h, eri = synth.hamiltonian(4, 8, seed=0)
    with pytest.raises(pkg.FnoccError):
        pkg.batch_solve([dict(h=h, eri=eri, nocc=8, threshold=1e-4)], ["ip"], 1)
    with pytest.raises(pkg.FnoccError):
        pkg.batch_solve([dict(h=h, eri=eri, nocc=2, threshold=1e-4)], [7], 1)
