"""Status codes of the C ABI on purpose: wrong call order (E_STATE), a NaN in
the input (E_NUMERIC), too few iterations (NOT_CONVERGED with every output
filled), bad arguments (E_INVALID), and the FNOCC_FAULT hook's failed
allocations (E_NOMEM), poisoned starting amplitude (E_NUMERIC) and
corrupted DIIS extrapolation. Every failure is made on the host side: a NaN
only travels through plain arithmetic kernels (no loop of any kernel
depends on the values), and the host detects it in the first energy; the
context stays usable afterwards.
"""
import ctypes
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

STATUS = {"E_INVALID": -1, "E_STATE": -4, "E_NUMERIC": -5, "NOT_CONVERGED": 1}


@pytest.fixture(scope="module")
def pkg():
    import paper_2509_14157_gb300 as p
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p.load_library()
    return p


def _status(pkg, fn, *a, **k):
    with pytest.raises(pkg.FnoccError) as ei:
        fn(*a, **k)
    return ei.value.status


def test_call_order(pkg):
    """ccsdt before a Hamiltonian, EOM and amplitudes before CCSDT, an EOM
    root before any EOM solve: E_STATE, and the context still works."""
    ctx = pkg.Context(0)
    lib = ctx.lib
    assert lib.ccsdt_solve(ctx._h, None, None) == STATUS["E_STATE"]
    assert b"Hamiltonian" in lib.fnocc_last_error(ctx._h)
    h, eri = synth.hamiltonian(4, 6, seed=0)
    ctx.fno_truncate(h, eri, 2, 0.0)
    assert _status(pkg, ctx.eom_solve, "ip", 2) == STATUS["E_STATE"]
    assert _status(pkg, ctx.get_block, "t1") == STATUS["E_STATE"]
    dim = sum(ctx.eom_sizes("ip"))
    assert _status(pkg, ctx.eom_sigma, "ip", np.zeros(dim)) == STATUS["E_STATE"]
    assert ctx.ccsdt_solve()["converged"]
    buf = np.zeros(1)
    assert lib.fnocc_get_block(ctx._h, 11, 0, buf.ctypes.data_as(pkg._dp), 1) == STATUS["E_STATE"]
    r = ctx.eom_solve("ip", 2)
    assert r["converged"] and np.all(np.isfinite(r["energies"]))
    ctx.close()


def test_nan_input_is_reported(pkg):
    """A NaN in the MO Hamiltonian: CCSDT stops with E_NUMERIC at its first
    energy; a clean Hamiltonian afterwards solves normally."""
    h, eri = synth.random_symmetric_mo_hamiltonian(6, 71)
    ctx = pkg.Context(0)
    bad = h.copy()
    bad[0, 0] = math.nan
    ctx.set_mo_hamiltonian(bad, eri, 2)
    assert _status(pkg, ctx.ccsdt_solve) == STATUS["E_NUMERIC"]
    assert b"NaN" in ctx.lib.fnocc_last_error(ctx._h)
    h0, eri0 = synth.hamiltonian(4, 6, seed=0)
    ctx.fno_truncate(h0, eri0, 2, 0.0)
    res = ctx.ccsdt_solve()
    assert res["converged"] and math.isfinite(res["e_corr"])
    ctx.close()


def test_not_converged_fills_outputs(pkg):
    """maxiter = 2: NOT_CONVERGED, with the last iterate's energies, sizes
    and amplitudes filled in (the binding returns converged = False)."""
    h, eri = synth.hamiltonian(4, 6, seed=0)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, 2, 0.0)
    lib = ctx.lib
    opt = pkg.CcsdtOptions(1e-10, 1e-12, 2, 8, 0, 1e-6)
    info = pkg.CcsdtInfo()
    st = lib.ccsdt_solve(ctx._h, ctypes.byref(opt), ctypes.byref(info))
    assert st == STATUS["NOT_CONVERGED"]
    # the energy of the second iterate (a large first Jacobi step can make it
    # positive; it only has to be the iterate's, finite and filled in)
    assert info.iters == 2 and math.isfinite(info.e_corr) and info.e_corr != 0.0 and info.res_max > 1e-10
    t2 = ctx.get_block("t2")
    assert np.all(np.isfinite(t2)) and np.max(np.abs(t2)) > 0
    res = ctx.ccsdt_solve(maxiter=2)
    assert not res["converged"]
    r = ctx.eom_solve("ip", 2, maxiter=2)
    assert not r["converged"]
    assert np.all(np.isfinite(r["energies"])) and np.all(r["energies"] != 0.0)
    assert r["iters"] <= 2
    ctx.close()


def test_bad_arguments(pkg):
    ctx = pkg.Context(0)
    h, eri = synth.hamiltonian(4, 6, seed=0)
    assert _status(pkg, ctx.fno_truncate, h, eri, 0, 1e-4) == STATUS["E_INVALID"]
    assert _status(pkg, ctx.fno_truncate, h, eri, 2, -1.0) == STATUS["E_INVALID"]
    ctx.fno_truncate(h, eri, 2, 0.0)
    ctx.ccsdt_solve()
    assert _status(pkg, ctx.eom_solve, 7, 2) == STATUS["E_INVALID"]
    assert _status(pkg, ctx.eom_solve, "ip", 0) == STATUS["E_INVALID"]
    assert ctx.lib.fnocc_set_precision(ctx._h, 9) == STATUS["E_INVALID"]
    ctx.close()


def test_fault_hook_alloc(pkg, monkeypatch):
    """FNOCC_FAULT=alloc: the device allocations of the FNO setup (the
    8-electron / 40-orbital integrals are 20 MB) fail as on a full device,
    E_NOMEM comes back through the ABI, and the same call succeeds once the
    variable is unset."""
    h, eri = synth.hamiltonian(8, 40, seed=0)
    ctx = pkg.Context(0)
    monkeypatch.setenv("FNOCC_FAULT", "alloc")
    assert _status(pkg, ctx.fno_truncate, h, eri, 4, 1e-4) == -2
    assert b"FNOCC_FAULT=alloc" in ctx.lib.fnocc_last_error(ctx._h)
    monkeypatch.delenv("FNOCC_FAULT")
    info = ctx.fno_truncate(h, eri, 4, 1e-4)
    assert info["nkept"] > 0
    ctx.close()


def test_fault_hook_nan_and_diverge(pkg, monkeypatch):
    """FNOCC_FAULT=nan: CCSDT starts from a NaN amplitude and stops with
    E_NUMERIC at its first energy. FNOCC_FAULT=diverge: every DIIS
    extrapolation is scaled by 1e3, and the solve ends in E_NUMERIC or
    NOT_CONVERGED. Unset, the same context converges to the undisturbed
    energy."""
    h, eri = synth.hamiltonian(6, 10, seed=0)
    ctx = pkg.Context(0)
    ctx.fno_truncate(h, eri, 3, 1e-4)
    ref = ctx.ccsdt_solve()
    assert ref["converged"]
    monkeypatch.setenv("FNOCC_FAULT", "nan")
    assert _status(pkg, ctx.ccsdt_solve) == STATUS["E_NUMERIC"]
    monkeypatch.setenv("FNOCC_FAULT", "diverge")
    try:
        res = ctx.ccsdt_solve(maxiter=60)
        assert not res["converged"]
    except pkg.FnoccError as e:
        assert e.status == STATUS["E_NUMERIC"]
    monkeypatch.delenv("FNOCC_FAULT")
    again = ctx.ccsdt_solve()
    assert again["converged"] and abs(again["e_corr"] - ref["e_corr"]) < 1e-10
    ctx.close()
