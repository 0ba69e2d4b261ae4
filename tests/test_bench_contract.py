"""Host test of bench.py's output contract (no GPU).

bench.main() runs against a stand-in library context and stand-ins for the
CUDA calls of torch, so only the script's own logic executes: the JSON line
must carry every key the benchmark contract names, with the arithmetic of
value, ms_per_step and the roofline fraction consistent, and the solver
statistics must be those of the timed FP64 steps (the mixed arm that runs
afterwards must not overwrite them). The reference arm's line is checked the
same way with its oracle sample replaced by a fixed stand-in.
"""
import json
import sys

import numpy as np
import pytest

import bench

torch = pytest.importorskip("torch")


class _Stream:
    cuda_stream = 0


class _Event:
    def __init__(self, **kw):
        self.t = 0.0

    def record(self, stream=None):
        import time
        self.t = time.perf_counter()

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


class FakeContext:
    """Stand-in for paper_2509_14157_gb300.Context: FP64 solves report 88
    products per variant, mixed ones 60."""
    PROFILE_PATHS = {}  # the real table, set by the fixture

    def __init__(self, *a, **k):
        self.launches, self.flops = 0, 0.0

    def profile(self, on):
        pass

    def profile_read(self, path):
        return (2.0, 1e9, 10) if path == 0 else (0.0, 0.0, 0)

    def fno_truncate_dev(self, *a, **k):
        return {"nkept": 15}

    def fno_truncate(self, h, eri, nocc, threshold, **k):
        return {"nkept": 15, "kept_fraction": threshold if 0 < threshold < 1 else 1.0}

    def ccsdt_solve(self, precision="fp64", **k):
        self.flops += 2e10
        self.launches += 100
        return dict(converged=True, iters=21, seconds=0.5, seconds_per_iter=0.02, e_corr=-0.3, e_tot=-21.3,
                    iters_mixed=0)

    def eom_solve(self, var, nroots, **kw):
        self.flops += 1e9
        self.launches += 50
        calls = 88 if kw.get("precision", "fp64") == "fp64" else 60
        return dict(energies=np.arange(nroots) * 0.1, omegas=np.arange(nroots) * 0.1, sigma_calls=calls,
                    iters=20, res_max=1e-9, complex_roots=0, seconds=0.1, seconds_per_iter=0.005,
                    converged=True, sigma_calls_mixed=0, guess_used=0)

    def set_guess_model(self, m):
        pass

    def dims(self):
        return 4, 8, -1.0

    # product-timing modes
    def amp_sizes(self):
        return [4, 6, 4]

    def set_amplitudes(self, *t):
        pass

    def set_precision(self, p):
        pass

    def eom_sizes(self, variant):
        return [2, 3, 4]

    def eom_sigma_dev(self, variant, x, s):
        self.calls = getattr(self, "calls", []) + [("right", variant)]

    def eom_left_sigma_dev(self, variant, x, s):
        self.calls = getattr(self, "calls", []) + [("left", variant)]

    def close(self):
        pass


class _Net:
    def close(self):
        pass


@pytest.fixture
def fake_gpu(monkeypatch):
    import paper_2509_14157_gb300 as pkg
    from paper_2509_14157_gb300 import learned
    real_device = torch.device
    monkeypatch.setattr(torch, "device", lambda *a, **k: real_device("cpu"))
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: _Stream())
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.cuda.nvtx, "range_push", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda.nvtx, "range_pop", lambda *a, **k: None)
    monkeypatch.setattr(FakeContext, "PROFILE_PATHS", dict(pkg.Context.PROFILE_PATHS))
    monkeypatch.setattr(pkg, "Context", FakeContext)

    def fake_batch_solve(systems, variants, nroots, nworkers=4, precision="fp64", **kw):
        om = np.zeros((len(systems), len(variants), nroots))
        info = [dict(status=0, nkept=4, e_rhf=-1.0, e_ccsdt=-1.1, ccsdt_iters=10, sigma_calls=50, seconds=0.1,
                     message="")
                for _ in systems]
        return om, info

    monkeypatch.setattr(pkg, "batch_solve", fake_batch_solve)
    monkeypatch.setattr(learned, "training_set", lambda *a, **k: (
        np.zeros((4, 8), np.float32), np.zeros((4, 2), np.float32), np.ones((4, 2), np.float32), [(0,)]))
    monkeypatch.setattr(learned, "train_guess_model", lambda *a, **k: (_Net(), [0.5]))
    seen = {}

    def fake_cpu_baseline(threshold, counts):
        seen["counts"] = counts
        return {"value": 100.0, "unit": "s", "cores": 1, "kind": "oracle", "sample": "stand-in"}

    class FakeSample:
        """Stand-in for the oracle sample: four work items, fixed estimate."""
        o, v = 4, 8

        def __init__(self, threshold):
            self.items = [("terms", ("residual", 1, 0), (0,))] * 3 + [("pack_t", None, None)]
            self.ran = 0

        def run(self, items):
            self.ran += len(items)
            seen["sample_items_run"] = self.ran

        def seconds_sampled(self):
            return 1.0

        def estimate(self, counts):
            seen["counts"] = counts
            return {"residual": 1.0, **{v: 1.0 for v in bench.VARIANTS}}, 100.0

    monkeypatch.setattr(bench, "cpu_baseline", fake_cpu_baseline)
    monkeypatch.setattr(bench, "OracleSample", FakeSample)
    monkeypatch.setattr(bench, "measured_fp64_peak", lambda device=0: (1.2, 1.0, "stand-in"))
    monkeypatch.setattr(bench, "NE", 2)      # small host arrays for the stand-in
    monkeypatch.setattr(bench, "NORB", 4)
    return seen


def _run(monkeypatch, capsys, argv):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    bench.main()
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_default_line_carries_the_contract(fake_gpu, monkeypatch, capsys):
    line = _run(monkeypatch, capsys, ["--steps", "2", "--warmup", "3"])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is False and line["scaling"] == "weak"
    assert "workload" in line["config"]
    assert abs(line["ms_per_step"] - 1e3 * line["value"] * len(bench.VARIANTS)) < 1e-9 * line["ms_per_step"]
    roof = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-12
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in line["cpu_baseline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in line["e2e"], key
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] > 0
    # statistics of the timed FP64 steps, not of the mixed arm that ran later
    assert line["solver"]["sigma_calls"] == {v: 88 for v in bench.VARIANTS}
    assert fake_gpu["counts"]["sigma"] == {v: 88 for v in bench.VARIANTS}
    assert line["mixed_learned"]["sigma_calls"] == {v: 60 for v in bench.VARIANTS}
    assert line["tflops"] > 0 and line["mixed_learned"]["tflops"] > 0


def test_reference_line_carries_the_contract(fake_gpu, monkeypatch, capsys):
    line = _run(monkeypatch, capsys, ["--impl", "reference", "--steps", "3", "--warmup", "2"])
    assert line["impl"] == "reference" and line["value"] == 100.0
    # the timed steps share the sample's work items: every item runs once, plus one per warm-up step
    assert fake_gpu["sample_items_run"] == 4 + 2
    assert line["ms_per_step"] >= 0 and line["config"]["precision"] == "fp64"
    for key in ("metric", "unit", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["e2e"] == {"value": 100.0, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert fake_gpu["counts"] is bench.REFERENCE_COUNTS


@pytest.mark.parametrize("argv,key", [(["--sigma-only", "dea"], "sigma_only"),
                                      (["--sigma-only", "ee", "--left"], "sigma_only"),
                                      (["--solve-only", "ee", "--left"], "solve_only"),
                                      (["--solve-only", "ip", "--precision", "mixed_tf32"], "solve_only"),
                                      (["--precision-check"], "mode"),
                                      (["--guess-check"], "mode"),
                                      (["--xfno-check"], "mode"),
                                      (["--batch"], "metric"),
                                      (["--batch", "--batch-large"], "metric")])
def test_timing_modes_run(fake_gpu, monkeypatch, capsys, argv, key):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    bench.main()
    lines = [json.loads(l) for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    line = lines[-1]
    assert key in line
    if key in ("sigma_only", "solve_only"):
        assert line[key] == argv[1] and line["left"] == ("--left" in argv) and line["seconds"] >= 0


def test_oracle_sample_covers_every_block_and_scales(monkeypatch):
    """The CPU baseline's sample: every Wick-term block of the residual and
    of every product has at least one sampled term (all of them at stride
    1), and the estimate scales each block's measured time by its term
    count and each residual / product by the given call counts."""
    monkeypatch.setattr(bench, "NE", 4)
    monkeypatch.setattr(bench, "NORB", 6)
    smp = bench.OracleSample(1e-4, stride=1)
    blocks = {it[1] for it in smp.items if it[0] == "terms"}
    assert blocks == set(smp.blocks)
    for kind, key, pick in smp.items:
        if kind == "terms":
            assert list(pick) == list(range(len(smp.blocks[key][0])))
    smp = bench.OracleSample(1e-4, stride=4)
    # injected times: every sampled block 2 s for m sampled terms (allocation 0)
    smp.times = {}
    for kind, key, pick in smp.items:
        if kind == "terms":
            smp.times[(kind, key)] = (0.0, 2.0, len(pick), len(smp.blocks[key][0]))
        else:
            smp.times[(kind, key)] = 0.5
    smp.t_fno = 1.0
    part_s, per_solve = smp.estimate({"cc_iters": 3, "sigma": {v: 10 for v in bench.VARIANTS}})
    res = sum(2.0 * len(smp.blocks[k][0]) / len([p for it in smp.items if it[1] == k for p in it[2]])
              for k in smp.blocks if k[0] == "residual") + 0.5
    assert abs(part_s["residual"] - res) < 1e-9
    step = 1.0 + 3 * part_s["residual"] + sum(10 * part_s[v] for v in bench.VARIANTS)
    assert abs(per_solve - step / len(bench.VARIANTS)) < 1e-9
