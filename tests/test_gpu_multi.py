"""Several volumes in one launch, CUDA-graph replay and the autotuner.

Each problem of a multi-volume step must follow the literal oracle
Algorithm 1 on its own batch (k mod n_batches), exactly as a single-problem
step would.
"""
import numpy as np
import pytest

import oracle as O
from cryo_cases import CTF_DICT, rel_l2
from paper_2311_16100_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM, BETA, CARM, K, SEED = 1e-2, 0.9, 0.5, 8, 77


class Dataset:
    """n_batches batches of B images of one volume (oracle forward + noise)."""

    def __init__(self, M, B, nb, seed):
        self.M, self.B, self.nb = M, B, nb
        n = B * nb
        self.r = M // 2 - 1
        self.vol = synth.blob_volume(M, seed=seed)
        self.quat = synth.shoemake_quaternions(n, seed + 1).astype(np.float32)
        self.R = O.quat_to_rot(self.quat.astype(np.float64)).astype(np.float32)
        self.df = synth.defocus_angstrom(n, seed + 2).astype(np.float32)
        clean = O.slice_project(self.vol, self.R, self.df, M, self.r, "trilinear", CTF_DICT)
        noise = synth.complex_normal((n, M, M), seed + 3, 0.05 * np.mean(np.abs(clean) ** 2))
        noise[:, ~O.disc_mask(M, self.r).reshape(M, M)] = 0
        self.images = (clean + noise).astype(np.complex64)
        self.alpha = O.alpha_threshold(self.df, M, self.r, CTF_DICT, LAM)
        self.v0 = (0.3 * self.vol).astype(np.complex64)

    def problem(self, ops, mode="hutchinson"):
        d = torch.device("cuda")
        geom = ops.Geometry(self.M, self.r, "trilinear", ops.CTF())
        st = ops.SGDState(torch.from_numpy(self.v0).to(d), mode=mode, alpha=self.alpha, eta0=4.0,
                          beta=BETA, armijo_c=CARM, n_probes=K, seed=SEED)
        self.t_images = torch.from_numpy(self.images).to(d)
        self.t_quat = torch.from_numpy(self.quat).to(d)
        self.t_df = torch.from_numpy(self.df).to(d)
        return ops.Problem(geom, st, self.t_images, self.t_quat, self.t_df, self.B, LAM,
                           float(self.nb))


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    h = ops.Handle(0)
    # 38: x rows of a length that is not a multiple of 4
    sets = [Dataset(24, 8, 2, 11), Dataset(32, 12, 2, 22), Dataset(38, 6, 3, 33)]
    yield ops, h, sets
    h.close()


def oracle_run(ds, steps, mode="hutchinson"):
    M = ds.M
    v, D, Da, eta = ds.v0.astype(np.complex128), np.ones((M, M, M)), np.zeros((M, M, M)), 4.0
    outs = []
    for k in range(1, steps + 1):
        b = (k - 1) % ds.nb
        sl = slice(b * ds.B, (b + 1) * ds.B)
        out = O.alg1_step(v, D, Da, eta, k, ds.images[sl], ds.R[sl], ds.df[sl], M, ds.r,
                          "trilinear", CTF_DICT, LAM, float(ds.nb), ds.alpha, BETA, CARM, mode,
                          n_probes=K, seed=SEED)
        v, D, Da, eta = out["v"], out["D"], out["D_avg"], out["eta"]
        outs.append(out)
    return outs


def test_multi_step_follows_oracle_per_problem(env):
    ops, h, sets = env
    probs = [ds.problem(ops) for ds in sets]
    steps = 4                       # wraps the 2-batch datasets
    ref = [oracle_run(ds, steps) for ds in sets]
    for k in range(steps):
        h.multi_step(probs)
        for p, ds in enumerate(sets):
            sc = probs[p].state.scalars.cpu().numpy()
            o = ref[p][k]
            assert sc[0] == o["eta"] and sc[6] == o["halvings"]
            assert abs(sc[3] - o["loss"]) <= 1e-5 * abs(o["loss"])
            assert rel_l2(probs[p].state.v.cpu().numpy(), o["v"]) <= 1e-4
            assert rel_l2(probs[p].state.D.cpu().numpy(), o["D"]) <= 1e-4
            assert sc[1] == k + 1


def test_multi_step_equals_single_problem_steps(env):
    ops, h, sets = env
    probs = [ds.problem(ops) for ds in sets]
    singles = [ds.problem(ops) for ds in sets]
    for k in range(3):
        h.multi_step(probs)
        for p, ds in enumerate(sets):
            b = k % ds.nb
            sl = slice(b * ds.B, (b + 1) * ds.B)
            q = singles[p]
            rot = h.quat_to_rot(q.quat[sl].contiguous())
            h.precond_sgd_step(q.geom, q.state, q.images[sl].contiguous(), rot,
                               q.defocus[sl].contiguous(), LAM, float(ds.nb))
    for a, b in zip(probs, singles):
        assert rel_l2(a.state.v.cpu().numpy(), b.state.v.cpu().numpy()) <= 1e-5
        assert float(a.state.scalars[0]) == float(b.state.scalars[0])


def test_graph_replay_matches_eager_steps(env):
    ops, h, sets = env
    eager = [ds.problem(ops) for ds in sets]
    graphed = [ds.problem(ops) for ds in sets]
    h2 = ops.Handle(0)             # a graph replays on its handle's workspace
    g = h2.multi_step_graph(graphed)
    s = torch.cuda.Stream()
    for _ in range(3):
        h.multi_step(eager)
        g.launch(s)
    torch.cuda.synchronize()
    for a, b in zip(eager, graphed):
        assert rel_l2(b.state.v.cpu().numpy(), a.state.v.cpu().numpy()) <= 1e-5
        assert float(a.state.scalars[1]) == float(b.state.scalars[1]) == 3.0
    g.close()
    h2.close()


def test_autotune_keeps_results(env):
    ops, h, sets = env
    probs = [ds.problem(ops) for ds in sets]
    before = [p.state.v.clone() for p in probs]
    bt, bps = h.autotune(probs)
    assert bt in (128, 256) and bps >= 1
    for p, v in zip(probs, before):          # state untouched by the tuner
        assert torch.equal(p.state.v, v) and float(p.state.scalars[1]) == 0.0
    ref = [oracle_run(ds, 1) for ds in sets]
    h.multi_step(probs)
    for p, ds in enumerate(sets):
        assert rel_l2(probs[p].state.v.cpu().numpy(), ref[p][0]["v"]) <= 1e-4
    h.set_launch_shape(256, 8)


def test_multi_step_rejects_mixed_modes(env):
    ops, h, sets = env
    from paper_2311_16100_gb300.ops import CryoSGDError
    probs = [sets[0].problem(ops, "hutchinson"), sets[1].problem(ops, "plain")]
    with pytest.raises(CryoSGDError):
        h.multi_step(probs)


def test_multi_step_with_slab_split_problems(env):
    """Problems whose grids are split into z-slabs (forced here with three
    slabs) run their own slab launches inside the multi-volume step: each
    problem still follows the oracle, eagerly and replayed as a graph."""
    ops, h, sets = env
    hs = ops.Handle(0)
    hs.set_slabs(3)
    probs = [ds.problem(ops) for ds in sets]
    ref = [oracle_run(ds, 2) for ds in sets]
    for k in range(2):
        hs.multi_step(probs)
        for p, ds in enumerate(sets):
            sc = probs[p].state.scalars.cpu().numpy()
            o = ref[p][k]
            assert sc[0] == o["eta"] and sc[6] == o["halvings"]
            assert abs(sc[3] - o["loss"]) <= 1e-5 * abs(o["loss"])
            assert rel_l2(probs[p].state.v.cpu().numpy(), o["v"]) <= 1e-4
    graphed = [ds.problem(ops) for ds in sets]
    eager = [ds.problem(ops) for ds in sets]
    hg = ops.Handle(0)
    hg.set_slabs(3)
    g = hg.multi_step_graph(graphed)
    for _ in range(2):
        hs.multi_step(eager)
        g.launch()
    torch.cuda.synchronize()
    for a, b in zip(eager, graphed):
        assert rel_l2(b.state.v.cpu().numpy(), a.state.v.cpu().numpy()) <= 1e-5
    g.close()
    hg.close()
    hs.close()
