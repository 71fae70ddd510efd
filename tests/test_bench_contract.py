"""The benchmark's JSON contract on the CPU side (no GPU): the CPU-baseline leg on a small
image, and the reference arm's line (keys, config identical to the GPU arm's, e2e with no
host-device bytes), with the oracle timing shortened."""
import argparse
import json

import numpy as np

import bench
import oracle as O
from paper_2405_02256_gb300 import synth


def test_cpu_baseline_on_a_small_image():
    """Two spawned processes on a small image: the keys the bench reports."""
    img = synth.grf((40, 48), 4.0, seed=3)
    dirs = synth.random_2d_dirs(16, 2, 0.01, 1.0)
    out = bench.cpu_baseline(img, synth.circle_dirs(8), dirs, budget_s=0.3, procs=2)
    assert out["kind"] == "oracle" and out["cores"] == 2 and out["nproc"] >= 1 and out["unit"] == bench.UNIT
    assert out["value"] > 0 and "40x48" in out["sample"]
    for key in ("ect_dirs_per_s", "radon_dirs_per_s", "tables_s_per_image"):
        assert out[key] > 0 and out["one_thread"][key] > 0
    assert out["one_thread"]["value"] > 0
    # the counted terms are the Delta-table sizes of the directions' orthants
    tab = O.critical_tables(img)
    assert all(len(tab.delta_idx[r]) > 0 for r in range(2))


def test_reference_arm_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "make_images", lambda count, side: [synth.grf((32, 32), 4.0, seed=1)])
    monkeypatch.setattr(bench, "cpu_baseline",
                        lambda img, dirs_e, dirs_h, budget_s=0.0: {"value": 123.0, "unit": bench.UNIT, "cores": 1,
                                                                   "kind": "oracle", "sample": "stub"})
    args = argparse.Namespace(images=64, side=2048, steps=2, warmup=3)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["config"] == bench.bench_config(64, 2048, 1)
    assert line["value"] == 123.0 and line["cpu_baseline"]["value"] == 123.0
    assert line["e2e"] == {"value": 123.0, "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["steps"] == 2 and line["warmup"] == 3


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setattr(bench, "_dist_info", lambda: (1, 2, 1))
    monkeypatch.setattr(bench, "make_images", lambda *a: (_ for _ in ()).throw(AssertionError("rank 1 worked")))
    bench.run_reference(None)
    assert capsys.readouterr().out == ""


def test_bench_config_names_the_workload():
    cfg = bench.bench_config(64, 2048, 1)
    assert cfg["images"] == 64 and cfg["side"] == 2048 and cfg["parallelism"] == "single GPU"
    assert "2048x2048" in cfg["workload"] and cfg["ht_dirs"] == 4096 and cfg["thresholds"] == 512
    assert bench.bench_config(64, 2048, 4)["parallelism"] == "replicas x4"
    assert np.isfinite(bench.whole_job_rate(1.0, 1, 1.0))
