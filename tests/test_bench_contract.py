"""The benchmark's reference arm (the FP64 oracle on the host) prints the
one-line JSON record of the benchmark contract; run on the CPU with a
one-image sample."""
import json
import os
import subprocess

import pytest
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cpu-sample", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
    assert d["cpu_baseline"]["kind"] == "oracle"
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    assert d["e2e"]["value"] == d["value"]


def test_disc_pixel_counts_and_job_value():
    """Disc pixel counts used for the algorithmic bytes and reductions (the
    disc kx^2 + ky^2 <= (M/2 - 1)^2: lattice points of a disc of radius r,
    counted row by row as sum over |ky| <= r of 2 floor(sqrt(r^2 - ky^2)) + 1),
    and the whole-job value (all ranks' images over the slowest rank's time)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import oracle as O
    import math
    for M in (32, 64, 128, 256):
        r = M // 2 - 1
        n = sum(2 * math.isqrt(r * r - ky * ky) + 1 for ky in range(-r, r + 1))
        assert bench.n_disc_pixels(M, r) == n
        assert int(np.count_nonzero(O.disc_mask(M, r))) == n
    assert [bench.n_disc_pixels(M, M // 2 - 1) for M in (32, 64, 128, 256)] == [709, 3001, 12453,
                                                                               50617]
    assert bench.job_value(4, 1024, 50, 1000.0) == 4 * 1024 * 50


def _stub_gpu_result():
    """A run_gpu result shaped like a real one (figures of a plausible run)."""
    roof = {"bound": "hbm", "kernel": "loss_grad", "achieved": 335.6, "peak": 6676.8,
            "unit": "GB/s", "frac": 0.0503, "peak_source": "measured", "traffic": 185700000,
            "algorithmic_bytes": 143970000, "ms_per_launch": 0.4291}
    red = {"bound": "l2_reductions", "kernel": "loss_grad", "achieved": 178.2, "peak": 207.6,
           "unit": "G reductions/s", "frac": 0.8584,
           "peak_source": "cs_measure_reduction_rate, live",
           "reductions_per_launch": 76507000}
    e2e = {"value": 1556000.0, "unit": "images/s", "h2d_bytes_per_step": 134238208,
           "d2h_bytes_per_step": 8, "host_wall_value": 1549000.0,
           "h2d_copy_only": {"GB_per_s": 211.3, "images_per_s_at_that_rate": 1610000.0},
           "direct_value": 1230000.0, "full_images_value": 1521000.0,
           "api": "cs_precond_sgd_step_host_disc (long description)"}
    return {"ms": 20 * 0.63, "timed_images": 20 * 1024, "launches": 220,
            "phases": {"precond": 0.02, "loss_grad": 0.429, "direction": 0.039,
                       "curvature": 0.136, "update": 0.019},
            "roofline": roof, "red_roofline": red, "e2e": e2e,
            "clocks": {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": [], "samples": 900,
                       "source": "nvml"},
            "scalars": [0.25, 25.0], "graph": {"images_per_s": 1623000.0},
            "loss_grad_only": {"value": 2620000.0}}


def _stub_race(arms):
    return {a: {"final_rel_err": 0.12345, "ms_to_rel_err": {"0.01": None if a == "plain"
                                                             else 139.4}} for a in arms}


def test_gpu_arm_record_is_compact_and_complete():
    """The GPU arm's last line (the contract record) carries every key the
    contract names and stays a few KB long, whatever the auxiliary legs
    produced (they are printed on earlier lines)."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=20, warmup=5, gpus=1, algo="auto")
    cfg = dict(bench.CONFIGS["m128"])
    tte = {"m32_nearest": _stub_race(["plain", "precomputed", "hutchinson"]),
           "m64_trilinear_ctf": _stub_race(["plain", "precomputed", "hutchinson"])}
    race64 = _stub_race(["plain", "precomputed", "hutchinson", "learned",
                         "exact_diagonal_control"])
    race64["setup_ms"] = {"learned": 1.234, "exact_diagonal_control": 4.56,
                          "precomputed": 78.9}
    learned = {"time_to_rel_err_64_snr10_b4096": race64}
    cpu = {"value": 72.6, "unit": "images/s", "cores": 16, "kind": "oracle",
           "sample": "one Algorithm-1 step of the FP64 numpy oracle per host core, "
                     "16 images each of the 128^3 workload, 16 single-threaded replicas "
                     "started together, 22.0 s wall",
           "sample_short": "FP64 oracle: one literal Algorithm-1 step of 16 images per core, "
                           "16 replicas, 22.0 s",
           "single_core": {"value": 10.8}, "operators_single_core": {"x": [1] * 500}}
    m2 = bench.metric2_summary(tte, learned)
    line = bench.contract_line(args, cfg, 1, _stub_gpu_result(), cpu, m2)
    text = json.dumps(line)
    # under 2 KB with room for the live figures' longer numbers
    assert len(text) < 1950, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "roofline_l2_reductions", "e2e", "cpu_baseline", "clocks",
              "gpu_launches", "metric2"):
        assert k in line, k
    assert line["value"] == round(20 * 1024 / (20 * 0.63e-3), 1)
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in line["cpu_baseline"], k
    assert "50000 images" in line["config"]["workload"]
    assert line["config"]["images_in_hbm_per_gpu"] == 50000
    assert set(m2) == {"m32_snr0.1", "m64_snr0.05", "m64_snr10_b4096"}
    # fixed-D arms carry their set-up time third; the others have none
    assert m2["m64_snr10_b4096"]["learned"] == [0.1235, 139.4, 1.2]
    assert m2["m64_snr10_b4096"]["pre"][2] == 78.9
    assert len(m2["m64_snr10_b4096"]["alg1"]) == 2 and len(m2["m32_snr0.1"]["pre"]) == 2
    assert len(json.dumps(m2)) < 600


def test_batches_cover_the_dataset_once():
    sys.path.insert(0, ROOT)
    import bench
    bl = bench.batches(50000, 1024)
    assert len(bl) == 49 and bl[-1] == (48 * 1024, 50000 - 48 * 1024)
    assert sum(n for _, n in bl) == 50000
    assert all(s == i * 1024 for i, (s, _) in enumerate(bl))
    assert bench.batches(1000, 100) == [(i * 100, 100) for i in range(10)]


def test_config_file_overrides_the_named_workload(tmp_path):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    f = tmp_path / "w.json"
    f.write_text(json.dumps({"M": 96, "n_img": 4096, "df": [0.5, 3.5], "snr": 0.2}))
    args = argparse.Namespace(config="m128", config_file=str(f), images=0)
    cfg = bench.workload_config(args)
    assert cfg["M"] == 96 and cfg["n_img"] == 4096 and cfg["df"] == (0.5, 3.5)
    assert cfg["B"] == bench.CONFIGS["m128"]["B"] and cfg["snr"] == 0.2
    f.write_text(json.dumps({"bogus": 1}))
    with pytest.raises(SystemExit):
        bench.workload_config(args)
    args = argparse.Namespace(config="m32", config_file=None, images=5000)
    assert bench.workload_config(args)["n_img"] == 5000
