"""The benchmark's reference arm (the FP64 oracle on the host) prints the
one-line JSON record of the benchmark contract; run on the CPU with a
one-image sample."""
import json
import os
import subprocess
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
