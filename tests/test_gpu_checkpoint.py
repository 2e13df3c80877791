"""Checkpoint / resume of Algorithm 1: the state saved after some steps and
restored into a fresh object continues the same trajectory (probes are
counter-based), matching an uninterrupted run."""
import numpy as np
import pytest

from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_resume_continues_the_same_trajectory(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    B, nb = 16, 3
    c = Case(32, B * nb, interp="trilinear", ctf=True, seed=95)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    h = ops.Handle(0)
    alpha = float(h.threshold_alpha(geom, g["df"], B * nb, 0.01))
    v0 = torch.from_numpy((0.3 * c.vol).astype(np.complex64)).cuda()

    def run(st, k0, k1):
        rot = torch.empty((B, 3, 3), device="cuda")
        for k in range(k0, k1):
            sl = slice((k % nb) * B, (k % nb + 1) * B)
            h.quat_to_rot(g["quat"][sl].contiguous(), rot)
            h.precond_sgd_step(geom, st, g["images"][sl].contiguous(), rot,
                               g["df"][sl].contiguous(), 0.01, float(nb))

    full = ops.SGDState(v0, mode="hutchinson", alpha=alpha, n_probes=8, seed=11)
    run(full, 0, 5)
    part = ops.SGDState(v0, mode="hutchinson", alpha=alpha, n_probes=8, seed=11)
    run(part, 0, 2)
    path = str(tmp_path / "state.pt")
    part.save(path)
    del part
    resumed = ops.SGDState.load(path)
    run(resumed, 2, 5)
    torch.cuda.synchronize()
    assert float(resumed.scalars[1]) == float(full.scalars[1]) == 5.0
    assert float(resumed.scalars[0]) == float(full.scalars[0])
    assert rel_l2(resumed.v.cpu().numpy(), full.v.cpu().numpy()) <= 1e-6
    assert rel_l2(resumed.D.cpu().numpy(), full.D.cpu().numpy()) <= 1e-6
    h.close()


def test_step_log_records_every_iteration(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import json
    from paper_2311_16100_gb300 import ops
    from paper_2311_16100_gb300.steplog import StepLog
    B, nb = 16, 2
    c = Case(32, B * nb, interp="trilinear", ctf=True, seed=96)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    h = ops.Handle(0)
    alpha = float(h.threshold_alpha(geom, g["df"], B * nb, 0.01))
    st = ops.SGDState(torch.from_numpy((0.3 * c.vol).astype(np.complex64)).cuda(),
                      mode="hutchinson", alpha=alpha, n_probes=8, seed=11)
    ref = g["vol"]
    path = str(tmp_path / "log.jsonl")
    log = StepLog(path, h, geom, reference=ref, flush_every=3)
    rot = torch.empty((B, 3, 3), device="cuda")
    for k in range(5):
        sl = slice((k % nb) * B, (k % nb + 1) * B)
        h.quat_to_rot(g["quat"][sl].contiguous(), rot)
        h.precond_sgd_step(geom, st, g["images"][sl].contiguous(), rot,
                           g["df"][sl].contiguous(), 0.01, float(nb))
        log.record(st)
    log.close()
    recs = [json.loads(line) for line in open(path)]
    assert [r["k"] for r in recs] == [1, 2, 3, 4, 5]
    assert recs[-1]["eta"] == float(st.scalars[0]) and all(r["status"] == 0 for r in recs)
    assert all(np.isfinite(r["loss"]) and r["loss"] > 0 for r in recs)
    final = float(h.rel_err(geom, st.v, ref))
    assert abs(recs[-1]["rel_err"] - final) <= 1e-12 * final
    h.close()
