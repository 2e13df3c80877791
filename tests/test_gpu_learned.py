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
