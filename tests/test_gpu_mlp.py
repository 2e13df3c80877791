"""Parity of the preconditioner network's kernels (tensor cores and FP32
reference) with the BF16-consistent FP64 oracle."""
import numpy as np
import pytest

from cryo_cases import rel_l2
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = (("W1", 0, 192, (64, 3)), ("b1", 192, 256, (64,)), ("W2", 256, 4352, (64, 64)),
         ("b2", 4352, 4416, (64,)), ("w3", 4416, 4480, (64,)), ("b3", 4480, 4481, (1,)))


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300.ops import Handle
    hd = Handle(0)
    yield hd
    hd.close()


def as_dict(flat):
    return {n: flat[a:b].astype(np.float64).reshape(shape) for n, a, b, shape in NAMES}


def inputs(M, seed):
    g = np.random.default_rng(seed)
    cov = g.uniform(0, 800, (M, M, M)).astype(np.float32)
    c2w = g.uniform(0, 300, (M, M, M)).astype(np.float32)
    tgt = g.normal(3.0, 1.0, (M, M, M)).astype(np.float32)
    from paper_2311_16100_gb300.learned import init_params
    return cov, c2w, tgt, init_params(seed)


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("M", [16, 22])
def test_forward_matches_oracle(h, tc, M):
    cov, c2w, _, P = inputs(M, M)
    d = torch.device("cuda")
    y = h.mlp_forward(M, torch.from_numpy(P).to(d), torch.from_numpy(cov).to(d),
                      torch.from_numpy(c2w).to(d), tensor_cores=tc)
    yo, _ = mlp.forward(as_dict(P), mlp.features(M, cov, c2w))
    assert rel_l2(y.cpu().numpy().ravel(), yo) <= 1e-3
    h.check_device_status()


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("M,r", [(16, 7), (22, 10)])
def test_gradient_matches_oracle(h, tc, M, r):
    cov, c2w, tgt, P = inputs(M, 100 + M)
    d = torch.device("cuda")
    grad = torch.zeros(4481, device=d)
    sse = torch.zeros((), dtype=torch.float64, device=d)
    h.mlp_grad(M, r, torch.from_numpy(P).to(d), torch.from_numpy(cov).to(d),
               torch.from_numpy(c2w).to(d), torch.from_numpy(tgt).to(d), grad, sse, tc)
    h.check_device_status()
    k = np.arange(M) - M // 2
    ball = ((k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2) <= r * r).ravel()
    X = mlp.features(M, cov, c2w)[ball]
    L, go = mlp.loss_and_grads(as_dict(P), X, tgt.ravel()[ball].astype(np.float64))
    g = grad.cpu().numpy()
    for n, a, b, shape in NAMES:
        assert rel_l2(g[a:b], go[n].ravel()) <= 1e-2, n
    assert abs(float(sse) / ball.sum() - L) <= 1e-4 * L


def test_tensor_core_and_reference_gradients_agree(h):
    M, r = 24, 11
    cov, c2w, tgt, P = inputs(M, 7)
    d = torch.device("cuda")
    args = [torch.from_numpy(a).to(d) for a in (P, cov, c2w, tgt)]
    out = []
    for tc in (True, False):
        grad = torch.zeros(4481, device=d)
        sse = torch.zeros((), dtype=torch.float64, device=d)
        h.mlp_grad(M, r, *args, grad, sse, tc)
        out.append(grad.cpu().numpy())
    for n, a, b, _ in NAMES:
        assert rel_l2(out[0][a:b], out[1][a:b]) <= 2e-3, n


def test_adam_step_matches_numpy(h):
    d = torch.device("cuda")
    g = np.random.default_rng(3)
    p = g.normal(size=4481).astype(np.float32)
    grad = g.normal(size=4481).astype(np.float32)
    tp, tg = torch.from_numpy(p).to(d), torch.from_numpy(grad).to(d)
    m, v = torch.zeros_like(tp), torch.zeros_like(tp)
    h.mlp_adam_step(tp, m, v, tg, 1, lr=0.01)
    # Adam, first step: m = (1-b1) g, v = (1-b2) g^2, bias-corrected update lr * g / (|g| + eps)
    mh = (1 - 0.9) * grad / (1 - 0.9)
    vh = (1 - 0.999) * grad ** 2 / (1 - 0.999)
    want = p - 0.01 * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(tp.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
    assert float(tg.abs().max()) == 0.0


def test_adam_gradient_scale_and_forward_offset(h):
    """The Adam step on grad_scale * grad equals the step on the scaled
    gradient; the forward's offset is added after exp (D = exp(net) + lambda)."""
    d = torch.device("cuda")
    g = np.random.default_rng(4)
    p = g.normal(size=4481).astype(np.float32)
    grad = g.normal(size=4481).astype(np.float32)
    a, b = torch.from_numpy(p).to(d), torch.from_numpy(p).to(d)
    ma, va, mb, vb = (torch.zeros_like(a) for _ in range(4))
    h.mlp_adam_step(a, ma, va, torch.from_numpy(grad).to(d), 1, lr=0.01, grad_scale=0.25)
    h.mlp_adam_step(b, mb, vb, torch.from_numpy(0.25 * grad).to(d), 1, lr=0.01)
    np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(ma.cpu().numpy(), mb.cpu().numpy(), rtol=1e-6, atol=1e-9)
    M = 16
    cov, c2w, _, P = inputs(M, 5)
    args = [torch.from_numpy(x).to(d) for x in (P, cov, c2w)]
    for tc in (True, False):
        y = h.mlp_forward(M, *args, tensor_cores=tc)
        D = h.mlp_forward(M, *args, exp=True, offset=2.5, tensor_cores=tc)
        np.testing.assert_allclose(D.cpu().numpy(), np.exp(y.cpu().numpy()) + 2.5, rtol=2e-6)
    from paper_2311_16100_gb300.ops import CryoSGDError
    with pytest.raises(CryoSGDError):
        h.mlp_forward(M, *args, offset=float("inf"))
    with pytest.raises(CryoSGDError):
        h.mlp_adam_step(a, ma, va, torch.zeros_like(a), 2, grad_scale=0.0)


def test_target_is_the_floored_log_mean_of_the_estimates(h):
    """cs_mlp_target: log(max(mean over estimates, floor x mean of the positive
    means)), written out in numpy."""
    d = torch.device("cuda")
    g = np.random.default_rng(6)
    M, n_est, floor = 20, 3, 0.05
    est = g.normal(5.0, 3.0, size=(n_est, M, M, M)).astype(np.float32)
    est[:, :2] = 0.0                      # some voxels unseen (mean 0)
    t = h.mlp_target(M, torch.from_numpy(est).to(d), floor).cpu().numpy()
    m = est.astype(np.float64).mean(axis=0)
    fl = floor * m[m > 0].mean()
    np.testing.assert_allclose(t, np.log(np.maximum(m, fl)), rtol=2e-6, atol=2e-6)
    assert float(t.min()) == pytest.approx(np.log(fl), rel=1e-5)
