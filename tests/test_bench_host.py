"""Host logic of bench.py on CPU: the time-to-tolerance protocol (stall
detection, the switch from the mixed to the FP64 form, E*, the first step
within 1e-6 Ha and its wall time) driven by a fake solver with prescribed
energy curves, and the scaling of the committed DRAM-traffic figures."""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

E_MIN = -10.0


def _curve(kind, start):
    """Energy after step k (k >= 1) of a run that starts from orbitals 'start'."""
    def e(k):
        if kind == "fp64":
            # converges geometrically to E_MIN from start
            return E_MIN + (start - E_MIN) * 0.995 ** k
        # mixed: fast, but stalls 5e-5 above the minimum
        return E_MIN + 5e-5 + (start - E_MIN - 5e-5) * 0.98 ** k
    return e


class FakeSolver:
    def __init__(self, precision):
        self.kind = "fp64" if precision == 0 else "mixed"
        self.E = []
        self.start = 0.0

    def set_atoms(self, *a):
        pass

    def set_orbitals(self, U):
        self.start = float(U)  # the fake "orbitals" are the energy they start from

    def iterate(self, n):
        f = _curve(self.kind, self.start)
        k0 = len(self.E)
        self.E.extend(f(k) for k in range(k0 + 1, k0 + n + 1))
        return {"energy": self.E[-1]}

    def history(self):
        return np.array(self.E), None

    def get_orbitals(self):
        return self.E[-1]

    def close(self):
        pass


def test_time_to_tolerance_protocol(monkeypatch):
    pou = types.SimpleNamespace(FP64=0, FP32=1)
    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    monkeypatch.setattr(bench, "make_solver", lambda pou, w, prec, stream, bb, **kw: FakeSolver(prec))
    clock = iter(np.arange(0.0, 1e6, 0.5))  # every perf_counter call advances 0.5 s
    monkeypatch.setattr(bench.time, "perf_counter", lambda: next(clock))
    args = types.SimpleNamespace(ttt_max=6000, ttt_fp64_max=4000, ttt_refine_max=6000, ttt_conv_rel=1e-10,
                                 ttt_ndiag=0, bb_variant=3, workload="fake")
    w = types.SimpleNamespace(width=0.8, name="fake")
    res = bench.time_to_tolerance(pou, torch, w, None, None, 0.0, types.SimpleNamespace(cuda_stream=0), args)
    # the mixed form stalls 5e-5 above the minimum: not reached, and it stopped early
    assert not res["mixed"]["reached"] and res["mixed"]["iterations"] < 6000
    assert res["mixed"]["final_error"] == pytest.approx(5e-5, rel=1e-3)
    # E* is the converged FP64 energy (the refined run gets within 1e-10 |E| per 100 steps)
    assert abs(res["E_star"] - E_MIN) < 1e-6
    # FP64 alone: first step within 1e-6 of E*, from a start 10 Ha above the minimum
    k = int(np.ceil(np.log(1e-6 / 10.0) / np.log(0.995)))
    assert res["fp64"]["reached"]
    assert abs(res["fp64"]["iterations"] - k) <= 1
    # the refined path: the switch happened at the stall, and it reached 1e-6 after the switch
    r = res["mixed_then_fp64"]
    assert r["reached"] and r["switched_at"]["mixed_steps"] == res["mixed"]["iterations"]
    assert r["iterations"] > r["switched_at"]["mixed_steps"]
    assert r["seconds"] > r["switched_at"]["seconds"] > 0.0


def test_traffic_scales_with_units_and_checks_the_source():
    t1 = bench.traffic_for("apply_h", 1000)
    if t1 is None:
        pytest.skip("no committed traffic entry for the current H-apply source")
    assert bench.traffic_for("apply_h", 2000) == pytest.approx(2 * t1)
    assert bench.traffic_for("no_such_kernel", 1000) is None


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the oracle, timed on a host core) prints one JSON
    line with the keys of the bench contract, for the workload it was given."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "l10_g32_n4"], capture_output=True, text=True, cwd=ROOT,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["metric"].startswith("outer iterations/s (32^3, N=4")
    assert d["config"]["workload"] == "l10_g32_n4"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert "all 4 orbitals" in d["cpu_baseline"]["sample"] and d["cpu_baseline"]["extrapolated"] is False
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["ms_per_step"] == pytest.approx(1e3 / d["value"])


def test_oracle_time_extrapolation_keeps_the_quadratic_term():
    """t(n) = a n + b n^2 recovered from two sample sizes and evaluated at N;
    a negative quadratic term from noisy samples is clamped to zero."""
    a, b = 0.4, 0.003
    t = lambda n: a * n + b * n * n
    per, a1, b1 = bench.extrapolate_iteration(t(8), 8, t(16), 16, 128)
    assert per == pytest.approx(t(128)) and a1 == pytest.approx(a) and b1 == pytest.approx(b)
    per, _, b2 = bench.extrapolate_iteration(3.3, 8, 6.5, 16, 128)
    assert b2 == 0.0 and per == pytest.approx(3.3 / 8 * 128)


def test_time_to_tolerance_refuses_caps_beyond_the_history():
    args = types.SimpleNamespace(ttt_max=20000, ttt_fp64_max=4000, ttt_refine_max=4000, ttt_conv_rel=1e-10,
                                 bb_variant=3, workload="fake")
    with pytest.raises(ValueError):
        bench.time_to_tolerance(None, None, types.SimpleNamespace(width=0.8, name="fake"), None, None, 0.0, None,
                                args)
