"""Oracle parity at launch shapes where every block of a grid walks several
work items, as the full-size runs do.

The small parity cases hold fewer work items than the traversal grid has
blocks (8 per SM), and fewer network tiles than the network kernels' grids,
so the loops over items and tiles run once per block there.  These cases
make them loop:
  * two Algorithm-1 steps at 64^3, batch 128, 32 probes, trilinear + CTF
    (about 2 000 items against the 1 216-block grid), through the default
    vector traversal and the three-slab one, against the literal oracle
    (Hutchinson with 32 separate Hessian-vector products, Armijo halving
    loop);
  * cs_hutchinson_diag at 128^3, batch 32, 32 probes;
  * the network's forward and gradient at 64^3 (2 048 tiles: 1.7 per CTA of
    the forward grid, 6.7 per CTA of the gradient grid) and the forward at
    128^3 (13.5 tiles per CTA) on a sample of voxels.
Tolerances as in the other parity tests (1e-4 gradient, diag and iterates;
1e-3 network forward and 1e-2 network gradient, BF16 operands).
"""
import numpy as np
import pytest

import oracle as O
from cryo_cases import Case, rel_l2
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
_ORACLE_STEPS = {}


def cpu(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=["vector", "vector_slabs3"])
def h(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300.ops import Handle
    hd = Handle(0)
    hd.set_algo("vector")
    if request.param == "vector_slabs3":
        hd.set_slabs(3)
    yield hd
    hd.close()


STEP = dict(M=64, B=128, nb=2, K=32, lam=1e-2, beta=0.9, carm=0.5, seed=41, eta0=4.0)


def _step_case():
    return Case(STEP["M"], STEP["B"] * STEP["nb"], interp="trilinear", ctf=True, seed=64)


def _oracle_steps(c, alpha):
    """The literal oracle's iterates for the two steps (computed once)."""
    if "steps" not in _ORACLE_STEPS:
        M, B = STEP["M"], STEP["B"]
        v = (0.3 * c.vol).astype(np.complex64).astype(np.complex128)
        D, Da, eta = np.ones((M, M, M)), np.zeros((M, M, M)), STEP["eta0"]
        outs = []
        for k in range(1, STEP["nb"] + 1):
            sl = slice((k - 1) * B, k * B)
            out = O.alg1_step(v, D, Da, eta, k, c.images[sl], c.R[sl], c.df[sl],
                              lam=STEP["lam"], scale=float(STEP["nb"]), alpha=alpha,
                              beta=STEP["beta"], c=STEP["carm"], mode="hutchinson",
                              n_probes=STEP["K"], seed=STEP["seed"], **c.geo())
            outs.append(out)
            v, D, Da, eta = out["v"], out["D"], out["D_avg"], out["eta"]
        _ORACLE_STEPS["steps"] = outs
    return _ORACLE_STEPS["steps"]


def test_alg1_steps_m64_b128_k32_follow_oracle(h):
    from paper_2311_16100_gb300.ops import SGDState
    c = _step_case()
    M, B = STEP["M"], STEP["B"]
    g = c.to_gpu()
    geom = c.gpu_geometry()
    alpha = O.alpha_threshold(c.df, M, c.r_max, c.ctf, STEP["lam"])
    v0 = (0.3 * c.vol).astype(np.complex64)
    st = SGDState(torch.from_numpy(v0).cuda(), mode="hutchinson", alpha=alpha,
                  eta0=STEP["eta0"], beta=STEP["beta"], armijo_c=STEP["carm"],
                  n_probes=STEP["K"], seed=STEP["seed"])
    outs = _oracle_steps(c, alpha)
    for k in range(1, STEP["nb"] + 1):
        sl = slice((k - 1) * B, k * B)
        h.precond_sgd_step(geom, st, g["images"][sl].contiguous(), g["rot"][sl].contiguous(),
                           g["df"][sl].contiguous(), STEP["lam"], float(STEP["nb"]))
        out = outs[k - 1]
        sc = cpu(st.scalars)
        assert sc[6] == out["halvings"] and sc[0] == out["eta"], (k, sc[0], out["eta"])
        assert abs(sc[3] - out["loss"]) <= 1e-5 * abs(out["loss"])
        assert rel_l2(cpu(st.v), out["v"]) <= TOL
        assert rel_l2(cpu(st.D), out["D"]) <= TOL
        assert rel_l2(cpu(st.D_avg), out["D_avg"]) <= TOL
        assert sc[1] == k


def test_hutchinson_diag_m128_b32_k32(h):
    c = Case(128, 32, interp="trilinear", ctf=True, seed=128)
    g = c.to_gpu()
    lam, scale = 0.05, 50000 / 32
    d = cpu(h.hutchinson_diag(c.gpu_geometry(), g["rot"], g["df"], lam, scale, n_probes=32,
                              seed=77, probe_block=5))
    dw = O.hutchinson_diag(c.R, c.df, lam=lam, scale=scale, n_probes=32, seed=77, block=5,
                           **c.geo())
    assert rel_l2(d, dw) <= TOL


NAMES = (("W1", 0, 192, (64, 3)), ("b1", 192, 256, (64,)), ("W2", 256, 4352, (64, 64)),
         ("b2", 4352, 4416, (64,)), ("w3", 4416, 4480, (64,)), ("b3", 4480, 4481, (1,)))


def _net_inputs(M, seed):
    g = np.random.default_rng(seed)
    cov = g.uniform(0, 800, (M, M, M)).astype(np.float32)
    c2w = g.uniform(0, 300, (M, M, M)).astype(np.float32)
    tgt = g.normal(3.0, 1.0, (M, M, M)).astype(np.float32)
    from paper_2311_16100_gb300.learned import init_params
    return cov, c2w, tgt, init_params(seed)


def _as_dict(flat):
    return {n: flat[a:b].astype(np.float64).reshape(shape) for n, a, b, shape in NAMES}


@pytest.fixture(scope="module")
def hn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300.ops import Handle
    hd = Handle(0)
    yield hd
    hd.close()


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("M,sample", [(64, None), (128, 40000)])
def test_network_forward_multi_tile(hn, tc, M, sample):
    cov, c2w, _, P = _net_inputs(M, 300 + M)
    d = torch.device("cuda")
    y = hn.mlp_forward(M, torch.from_numpy(P).to(d), torch.from_numpy(cov).to(d),
                       torch.from_numpy(c2w).to(d), tensor_cores=tc)
    hn.check_device_status()
    X = mlp.features(M, cov, c2w)
    idx = (np.arange(M ** 3) if sample is None
           else np.random.default_rng(M).choice(M ** 3, size=sample, replace=False))
    yo, _ = mlp.forward(_as_dict(P), X[idx])
    assert rel_l2(y.cpu().numpy().ravel()[idx], yo) <= 1e-3


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("M", [250, 510])
def test_network_forward_large_grid_sampled(hn, tc, M):
    """Grids whose voxel indices exceed 2^24 (510^3) or are not powers of two
    (250): the kernels take a voxel's coordinates from a float reciprocal of
    M with one correction step; 40 000 sampled voxels against the oracle."""
    g = np.random.default_rng(500 + M)
    cov = (g.random((M, M, M), dtype=np.float32) * 800).astype(np.float32)
    c2w = (g.random((M, M, M), dtype=np.float32) * 300).astype(np.float32)
    from paper_2311_16100_gb300.learned import init_params
    P = init_params(M)
    d = torch.device("cuda")
    y = hn.mlp_forward(M, torch.from_numpy(P).to(d), torch.from_numpy(cov).to(d),
                       torch.from_numpy(c2w).to(d), tensor_cores=tc)
    hn.check_device_status()
    # the sample includes the grid's last voxels (the largest indices)
    idx = np.concatenate([g.choice(M ** 3, size=40000, replace=False),
                          np.arange(M ** 3 - 256, M ** 3)])
    yo, _ = mlp.forward(_as_dict(P), mlp.features(M, cov, c2w, idx))
    assert rel_l2(y.cpu().numpy().ravel()[idx], yo) <= 1e-3


@pytest.mark.parametrize("tc", [True, False])
def test_network_gradient_multi_tile(hn, tc):
    M, r = 64, 31
    cov, c2w, tgt, P = _net_inputs(M, 400)
    d = torch.device("cuda")
    grad = torch.zeros(4481, device=d)
    sse = torch.zeros((), dtype=torch.float64, device=d)
    hn.mlp_grad(M, r, torch.from_numpy(P).to(d), torch.from_numpy(cov).to(d),
                torch.from_numpy(c2w).to(d), torch.from_numpy(tgt).to(d), grad, sse, tc)
    hn.check_device_status()
    k = np.arange(M) - M // 2
    ball = ((k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
            <= r * r).ravel()
    X = mlp.features(M, cov, c2w)[ball]
    L, go = mlp.loss_and_grads(_as_dict(P), X, tgt.ravel()[ball].astype(np.float64))
    gg = grad.cpu().numpy()
    for n, a, b, shape in NAMES:
        assert rel_l2(gg[a:b], go[n].ravel()) <= 1e-2, n
    assert abs(float(sse) / ball.sum() - L) <= 1e-4 * L
