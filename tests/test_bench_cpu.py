"""The bench's host-side pieces (no GPU): the reference arm's JSON line
(the oracle timed on the host cores) keeps the contract's keys, and the
oracle baselines of the NDFD and point-feature workloads run on host
tensors."""
import json
import os
import subprocess
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "20000"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_ndfd_and_point_oracle_baselines_on_host_tensors():
    import bench
    from paper_2505_19154_gb300 import synth
    scene, cams = synth.config3(0, n=20000, D=0)
    feats, fgt = synth.ndfd_inputs_device(0, 20000, cams, 32, torch.device("cpu"))
    P = fgt.shape[0]
    r = bench.ndfd_cpu_baseline(scene, cams, feats, fgt, torch.randn(P), torch.randn(P), max_seconds=2, reps_max=1)
    assert r["kind"] == "oracle" and r["value"] > 0 and "NDFD" in r["sample"]
    sc5, views = synth.config5(0, n=50000)
    views = views[:4]
    means = torch.from_numpy(np.ascontiguousarray(sc5["means"], np.float32))
    maps = [torch.zeros((v["height"] * v["width"], 8)) for v in views]
    r = bench.points_cpu_baseline(means, views, maps, torch.rand(means.shape[0]))
    assert r["kind"] == "oracle" and r["value"] > 0


def test_cpu_baseline_runs_the_reference_arm_in_a_fresh_process():
    import bench
    r = bench.cpu_baseline(20_000, 16, steps=1, warmup=1)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1, r
    assert "fresh process" in r["sample"]
