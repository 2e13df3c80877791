"""What the learned preconditioner gains over Algorithm 1 without it.

The network is trained (on the GPU, by the library's kernels) on Hutchinson
estimates of diag(H) from four datasets and applied to a fifth, unseen one.
Compared there: its D against the exact diagonal, against Algorithm 1's
running estimate after one epoch (which starts from D = I), and the
relative volume error of SGD preconditioned by each after one epoch.
"""
import numpy as np
import pytest

from cryo_cases import rel_l2
from paper_2311_16100_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, N, B = 32, 2000, 100
R_MAX = M // 2 - 1


def dataset(h, ops, seed, with_images=False):
    quat = synth.shoemake_quaternions(N, seed + 1).astype(np.float32)
    d = torch.device("cuda")
    rot = h.quat_to_rot(torch.from_numpy(quat).to(d))
    df = torch.from_numpy(synth.defocus_angstrom(N, seed + 2, 0.5, 3.5).astype(np.float32)).to(d)
    return rot, df


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    from paper_2311_16100_gb300.learned import (LearnedPreconditioner, Sample, dataset_features,
                                                hutchinson_target)
    h = ops.Handle(0)
    geom = ops.Geometry(M, R_MAX, "trilinear", ops.CTF())
    samples = []
    for s in range(4):
        rot, df = dataset(h, ops, 4000 + 10 * s)
        cov, c2w = dataset_features(h, geom, rot, df)
        samples.append(Sample(M, R_MAX, cov, c2w, hutchinson_target(h, geom, rot, df)))
    net = LearnedPreconditioner(h, seed=1)
    hist = net.fit(samples, steps=400, lr=1e-2)
    yield ops, h, geom, net, hist
    h.close()


def test_training_reduces_the_loss(trained):
    _, _, _, _, hist = trained
    assert hist[-1] < 0.05 * hist[0]


def test_learned_D_beats_one_epoch_of_algorithm_1(trained):
    ops, h, geom, net, _ = trained
    rot, df = dataset(h, ops, 9000)
    lam = 1.0
    exact, _, _ = h.exact_diag(geom, rot, df, lam, 1.0)
    from paper_2311_16100_gb300.learned import dataset_features
    cov, c2w = dataset_features(h, geom, rot, df)
    D_learned = net.predict(M, cov, c2w, lam)
    ball = torch.from_numpy(synth.ball_mask(M, R_MAX)).cuda()
    err_learned = rel_l2(D_learned[ball].cpu().numpy(), exact[ball].cpu().numpy())
    # Algorithm 1's estimate after one epoch: D^(k) = beta D^(k-1) + (1-beta) D_avg
    D = torch.ones_like(exact)
    Davg = torch.zeros_like(exact)
    for k in range(1, N // B + 1):
        sl = slice((k - 1) * B, k * B)
        dest = h.hutchinson_diag(geom, rot[sl].contiguous(), df[sl].contiguous(), lam, N / B,
                                 n_probes=32, seed=5, probe_block=k)
        Davg = (k - 1) / k * Davg + dest / k
        D = 0.9 * D + 0.1 * Davg
    err_alg1 = rel_l2(D[ball].cpu().numpy(), exact[ball].cpu().numpy())
    assert err_learned < 0.25
    assert err_learned < err_alg1


# ------------------------------------------------------------------ 64^3
M64, N64, B64, SUB = 64, 8192, 1024, 8


def _cg(h, geom, rot, df, b, lam, iters=300):
    """v* = H^{-1} b (full-data Hessian) by conjugate gradients through the
    library's gradient (H p = grad of the loss at p with zero images)."""
    zeros = torch.zeros((rot.shape[0], geom.M, geom.M), dtype=torch.complex64, device="cuda")
    x = torch.zeros_like(b)
    r = b.clone()
    p = r.clone()
    rs = float(torch.sum(torch.abs(r) ** 2))
    bn = rs ** 0.5
    for _ in range(iters):
        _, Hp = h.loss_grad(geom, p, zeros, rot, df, lam, 1.0)
        a = rs / float(torch.sum((torch.conj(p) * Hp).real))
        x += a * p
        r -= a * Hp
        rs_new = float(torch.sum(torch.abs(r) ** 2))
        if rs_new ** 0.5 <= 1e-6 * bn:
            break
        p = r + (rs_new / rs) * p
        rs = rs_new
    return x


@pytest.fixture(scope="module")
def trained64():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    from paper_2311_16100_gb300.learned import (LearnedPreconditioner, Sample, dataset_features,
                                                hutchinson_target)
    h = ops.Handle(0)
    r = M64 // 2 - 1
    geom = ops.Geometry(M64, r, "trilinear", ops.CTF())
    d = torch.device("cuda")
    sets = []
    for s in range(5):
        q = torch.from_numpy(synth.shoemake_quaternions(N64, 6400 + 10 * s)
                             .astype(np.float32)).to(d)
        df = torch.from_numpy(synth.defocus_angstrom(N64, 6401 + 10 * s, 0.5, 3.5)
                              .astype(np.float32)).to(d)
        sets.append((h.quat_to_rot(q), df))
    samples = []
    for rot, df in sets[:4]:
        cov, c2w = dataset_features(h, geom, rot, df, subsample=SUB)
        samples.append(Sample(M64, r, cov, c2w, hutchinson_target(h, geom, rot, df)))
    net = LearnedPreconditioner(h, seed=2)
    net.fit(samples, steps=300, lr=1e-2)
    yield ops, h, geom, net, sets[4]
    h.close()


def test_learned_preconditioner_gains_at_64(trained64):
    """On a fifth, unseen pose set at 64^3 (8192 poses, trilinear, CTF), the
    network trained on four others, with features from one eighth of the
    poses, is compared with Algorithm 1 (D^(0) = I) and with the exact
    diagonal (cs_exact_diag, one pass over all poses):
      * its D is within 25% (relative L2 over the ball) of the exact diagonal
        and closer to it than Algorithm 1's D after one epoch;
      * SGD preconditioned by it reaches a lower relative error against v*
        after two epochs (SNR 10, batch 1024) than Algorithm 1;
      * its set-up (feature pass over one eighth of the poses + inference)
        takes less device time than the exact diagonal's pass."""
    from paper_2311_16100_gb300.learned import dataset_features
    ops, h, geom, net, (rot, df) = trained64
    d = torch.device("cuda")
    r = M64 // 2 - 1
    ball = torch.from_numpy(synth.ball_mask(M64, r)).to(d)
    v_true = torch.from_numpy(synth.blob_volume(M64, seed=6500)).to(d)
    clean = h.slice_project(geom, v_true, rot, df)
    disc = ball[M64 // 2]
    sig2 = float((clean.abs() ** 2)[:, disc].mean()) / 10.0
    gen = torch.Generator(device=d)
    gen.manual_seed(6501)
    noise = torch.randn(clean.shape, dtype=torch.complex64, device=d, generator=gen)
    images = clean + noise * (sig2 ** 0.5) * disc.to(torch.complex64)
    lam = sig2
    # set-up times (device), then the preconditioners
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):                                    # second round timed
        torch.cuda.synchronize()
        e0.record()
        cov, c2w = dataset_features(h, geom, rot, df, subsample=SUB)
        D_learned = net.predict(M64, cov, c2w, lam)
        e1.record()
        torch.cuda.synchronize()
        t_learned = e0.elapsed_time(e1)
        e0.record()
        exact, _, _ = h.exact_diag(geom, rot, df, lam, 1.0)
        e1.record()
        torch.cuda.synchronize()
        t_exact = e0.elapsed_time(e1)
    err_learned = rel_l2(D_learned[ball].cpu().numpy(), exact[ball].cpu().numpy())
    D = torch.ones_like(exact)
    Davg = torch.zeros_like(exact)
    for k in range(1, N64 // B64 + 1):
        sl = slice((k - 1) * B64, k * B64)
        dest = h.hutchinson_diag(geom, rot[sl].contiguous(), df[sl].contiguous(), lam,
                                 N64 / B64, n_probes=32, seed=5, probe_block=k)
        Davg = (k - 1) / k * Davg + dest / k
        D = 0.9 * D + 0.1 * Davg
    err_alg1_D = rel_l2(D[ball].cpu().numpy(), exact[ball].cpu().numpy())
    # SGD from the same start, same batches: learned D vs Algorithm 1
    b = h.backproject_adjoint(geom, images, rot, df, 1.0)
    vstar = torch.where(ball, _cg(h, geom, rot, df, b, lam), torch.zeros_like(b))
    alpha = h.threshold_alpha(geom, df, N64, lam)
    v0 = torch.from_numpy(synth.initial_volume(M64, r, 1.0, 6502)).to(d)
    errs = {}
    for name, mode, Dinit in (("learned", "fixed", D_learned), ("alg1", "hutchinson", None)):
        st = ops.SGDState(v0, mode=mode, alpha=alpha, eta0=1.0, beta=0.9, armijo_c=0.5,
                          n_probes=32, seed=7, D=Dinit)
        for ep in range(2):
            perm = torch.from_numpy(synth.permutation(N64, 6503 + ep)).to(d)
            xp, rp, dp = images[perm].contiguous(), rot[perm].contiguous(), df[perm].contiguous()
            for s in range(0, N64, B64):
                h.precond_sgd_step(geom, st, xp[s:s + B64], rp[s:s + B64], dp[s:s + B64], lam,
                                   N64 / B64)
        errs[name] = float(h.rel_err(geom, st.v, vstar))
    print(f"\nlearned D error {err_learned:.4f} (Algorithm 1 after one epoch {err_alg1_D:.4f}); "
          f"SGD rel. error after 2 epochs: learned {errs['learned']:.4f}, "
          f"Algorithm 1 {errs['alg1']:.4f}; set-up {t_learned:.3f} ms vs exact diagonal "
          f"{t_exact:.3f} ms")
    assert err_learned < 0.25 and err_learned < err_alg1_D
    assert errs["learned"] < errs["alg1"]
    assert t_learned < t_exact
