"""Full-size launches against the oracle on sampled voxels.

The benchmark's own launch (128^3, batch 1024, trilinear + CTF, 32 probes)
and the z-slab traversal of a 256^3 grid (batch 64) are checked against the
FP64 oracle where it can be evaluated: Hutchinson's estimate at 32 sampled
voxels of the ball (oracle.hutchinson_diag_at: the literal K-probe sum for
those rows), the Algorithm-1 step's running mean D_avg (the same estimate at
k = 1) and its update v - eta g / D-hat at those voxels (the oracle's full
gradient), the batch loss, and the accepted eta against the closed-form
Armijo bound from the oracle's G and Q (reading 11).
"""
import numpy as np
import pytest

import oracle as O
from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def cpu(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("M,B", [(128, 1024), (256, 64)])
def test_full_size_step_on_sampled_voxels(M, B):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300.ops import Handle, SGDState
    c = Case(M, B, interp="trilinear", ctf=True, seed=4000 + M)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    h = Handle(0)
    N = 50 * B                                  # the mini-batch's scale N / |I|
    lam, scale, K, seed, beta, carm = 1e-2, float(N) / B, 32, 5, 0.9, 0.5
    rng = np.random.default_rng(M)
    ball = np.nonzero(O.ball_mask(M, c.r_max))[0]
    centre = ((M // 2) * M + M // 2) * M + M // 2
    sel = np.unique(np.concatenate([rng.choice(ball, size=31, replace=False), [centre + 1]]))
    want = O.hutchinson_diag_at(sel, c.R, c.df, lam=lam, scale=scale, n_probes=K, seed=seed,
                                block=1, **c.geo())
    # the Hutchinson entry point (pixel kernel)
    d = cpu(h.hutchinson_diag(geom, g["rot"], g["df"], lam, scale, n_probes=K, seed=seed,
                              probe_block=1)).ravel()
    assert rel_l2(d[sel], want) <= TOL
    # one Algorithm-1 step (the fused traversal; z-slabs at 256^3)
    alpha = float(np.median(want))
    v0 = (0.5 * c.vol).astype(np.complex64)
    st = SGDState(torch.from_numpy(v0).cuda(), mode="hutchinson", alpha=alpha, eta0=4.0,
                  beta=beta, armijo_c=carm, n_probes=K, seed=seed)
    h.precond_sgd_step(geom, st, g["images"], g["rot"], g["df"], lam, scale)
    sc = cpu(st.scalars)
    assert rel_l2(cpu(st.D_avg).ravel()[sel], want) <= TOL
    f, grad = O.loss_grad(v0, c.images, c.R, c.df, lam=lam, scale=scale, **c.geo())
    assert abs(sc[3] - f) <= 1e-5 * abs(f)
    dhat = np.maximum(np.abs(beta + (1 - beta) * want), alpha)
    eta = sc[0]
    assert eta == 4.0 * 2.0 ** (-sc[6])
    v_want = v0.ravel()[sel] - eta * grad.ravel()[sel] / dhat
    assert rel_l2(cpu(st.v).ravel()[sel], v_want) <= TOL
    # the accepted eta is the first halving under the Armijo bound (G, Q
    # from the oracle, with the step's own D-hat, checked above at samples)
    Dh = np.maximum(np.abs(cpu(st.D)).astype(np.float64), alpha)
    dd = grad / Dh
    G = float(np.sum(np.abs(grad) ** 2 / Dh))
    Pd = O.slice_project(dd, c.R, c.df, **c.geo())
    Q = scale * float(np.sum(np.abs(Pd) ** 2)) + lam * float(np.sum(np.abs(dd) ** 2))
    bound = 2 * (1 - carm) * G / Q
    assert eta <= bound * (1 + 1e-5)
    assert eta == 4.0 or 2 * eta > bound * (1 - 1e-5)
    h.close()
