"""bench.py host logic without a GPU: the `forms` summary of the default line
(the batching and serving runs in child processes) is built from their JSON lines,
and a child that fails, times out or prints something unexpected leaves an error
entry instead of taking the headline line down."""
import json
import subprocess
import types

import pytest

import bench


def _child_line(name):
    line = {"value": 2.0e11, "unit": "samples/s", "ms_per_step": 500.0, "steps": 3,
            "e2e": {"value": 1.9e11, "ms_per_step": 520.0}, "roofline": {"frac": 0.5, "kernel_ms": 490.0},
            "gpu_launches": 80, "clocks": {"sm_mhz": 2070.0}, "config": {"autotuned": {"lanes_per_contour": 8}}}
    if name == "batch-3d":
        line["detection"] = {"f": 0.88}
    else:
        line["serving"] = {"saturated_latency_ms_p50": 470.0, "latency_ms_p50": 52.0, "latency_ms_p99": 130.0,
                           "poisson_lambda_hz": 24.8, "saturated_tiles_per_s": 35.0,
                           "budget_bound_saturated": {"budget_gb": 0.4}}
    return json.dumps(line)


def _fake(monkeypatch, behave):
    def run(cmd, capture_output, text, timeout):
        name = cmd[cmd.index("--workload") + 1]
        return behave(name, cmd, timeout)
    monkeypatch.setattr(bench.subprocess, "run", run)


def test_forms_summary(monkeypatch):
    seen = []

    def behave(name, cmd, timeout):
        seen.append(cmd)
        return types.SimpleNamespace(returncode=0, stdout="log line\n" + _child_line(name) + "\n", stderr="")
    _fake(monkeypatch, behave)
    out = bench.run_forms()
    assert set(out) == {"batch-3d", "serve-3d"}
    b, s = out["batch-3d"], out["serve-3d"]
    assert b["value"] == 2.0e11 and b["e2e"]["value"] == 1.9e11 and b["evolve_kernel_ms"] == 490.0
    assert b["detection_f"] == 0.88 and b["autotuned"] == {"lanes_per_contour": 8}
    assert s["latency_ms"] == {"saturated_p50": 470.0, "poisson_p50": 52.0, "poisson_p99": 130.0,
                               "poisson_lambda_hz": 24.8}
    assert s["saturated_tiles_per_s"] == 35.0 and s["budget_bound"] == {"budget_gb": 0.4}
    assert all("--no-cpu-baseline" in c for c in seen)
    assert b["command"].endswith("--steps 3 --warmup 3")


@pytest.mark.parametrize("mode", ["exit", "timeout", "garbage", "missing_key"])
def test_forms_failures_leave_an_error_entry(monkeypatch, mode):
    def behave(name, cmd, timeout):
        if mode == "exit":
            return types.SimpleNamespace(returncode=1, stdout="", stderr="CUDA error: out of memory")
        if mode == "timeout":
            raise subprocess.TimeoutExpired(cmd, timeout)
        if mode == "garbage":
            return types.SimpleNamespace(returncode=0, stdout="not json", stderr="")
        d = json.loads(_child_line(name))
        del d["roofline"]
        return types.SimpleNamespace(returncode=0, stdout=json.dumps(d), stderr="")
    _fake(monkeypatch, behave)
    out = bench.run_forms()
    for name in ("batch-3d", "serve-3d"):
        assert set(out[name]) == {"error"}, out[name]
    if mode == "exit":
        assert "out of memory" in out["batch-3d"]["error"]
