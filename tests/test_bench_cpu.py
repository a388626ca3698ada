"""bench.py, smoke() and the binding on a machine without a GPU.

* The reference arm (the oracle timed on the host cores) returns the JSON line
  of the benchmark contract: metric, value and unit of the GPU arm, its CPU
  baseline with the single-thread rate beside it, and an end-to-end block with
  no host-device copies.
* Without CUDA the GPU arm of bench.py, smoke() and the binding fail loudly:
  there is no CPU fallback on the product path.
"""

import json
import os
import subprocess
import sys
from types import SimpleNamespace

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

no_cuda = pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without CUDA")


def test_reference_arm_line(monkeypatch):
    import bench

    full = bench.cpu_oracle_rate
    # a short sample: the line's shape is under test here, not the rate
    monkeypatch.setattr(bench, "cpu_oracle_rate", lambda seed, budget_s=0.3: full(seed, budget_s=0.3))
    line = bench.run_reference(SimpleNamespace(steps=1, warmup=0), 1, 0)
    json.dumps(line)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["metric"].startswith("all-pairs DTW GCUPS") and line["unit"] == "GCUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["single_thread"]["value"] > 0 and cb["single_thread"]["unit"] == "GCUPS"
    assert line["e2e"] == {"value": line["value"], "unit": "GCUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    import bench

    assert bench.run_reference(SimpleNamespace(steps=1, warmup=0), 2, 1) is None


@no_cuda
def test_gpu_arm_fails_without_cuda():
    r = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "3",
                        "--no-cpu-baseline"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0
    for ln in r.stdout.splitlines():  # no measurement line of the GPU arm
        try:
            assert json.loads(ln).get("impl") != "dtwgb"
        except ValueError:
            pass


@no_cuda
def test_smoke_fails_without_cuda():
    r = subprocess.run([sys.executable, "-c", "import __graft_entry__ as g; g.smoke()"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0


@no_cuda
def test_binding_refuses_host_tensors():
    from paper_2307_04904_gb300 import api

    v = torch.zeros(10, dtype=torch.float32)
    o = torch.tensor([0, 5, 10], dtype=torch.int64)
    with pytest.raises((TypeError, RuntimeError)):
        api.dtw_pairwise(v, o, 2)
    with pytest.raises((TypeError, RuntimeError)):
        api.kmedoids_fit(torch.zeros((4, 4)), 2, torch.tensor([0, 1], dtype=torch.int32))
