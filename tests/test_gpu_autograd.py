"""The autograd Function: its backward is the library's adjoint kernel.

Checked against central finite differences of L = 1/2 |C P v - x|^2 on
random voxels (exact for a quadratic up to rounding; h = 1e-3) and against
the FP64 oracle gradient, at the 128^3, 1024-image size and on small cases.
"""
import numpy as np
import pytest

import oracle as O
from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda")


def _loss64(y, x):
    return 0.5 * float(torch.sum(torch.abs(y.to(torch.complex128) - x.to(torch.complex128)) ** 2))


@pytest.mark.parametrize("M,B", [(32, 40), (128, 1024)])
def test_backward_matches_oracle_gradient(dev, M, B):
    from paper_2311_16100_gb300.autograd import slice_project
    c = Case(M, B, interp="trilinear", ctf=True, seed=5000 + M)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    v = g["vol"].clone().requires_grad_(True)
    y = slice_project(v, g["rot"], g["df"], geom)
    L = 0.5 * torch.sum(torch.abs(y - g["images"]) ** 2)
    L.backward()
    _, gw = O.loss_grad(c.vol, c.images, c.R, c.df, lam=0.0, scale=1.0, **c.geo())
    assert rel_l2(v.grad.detach().cpu().numpy(), gw) <= 1e-4


@pytest.mark.parametrize("M,B", [(32, 40), (128, 1024)])
def test_backward_matches_central_differences(dev, M, B):
    from paper_2311_16100_gb300.autograd import slice_project
    c = Case(M, B, interp="trilinear", ctf=True, seed=6000 + M)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    v = (0.5 * g["vol"]).clone().requires_grad_(True)
    y = slice_project(v, g["rot"], g["df"], geom)
    L = 0.5 * torch.sum(torch.abs(y - g["images"]) ** 2)
    L.backward()
    grad = v.grad.detach()
    rng = np.random.default_rng(M)
    ball = np.flatnonzero(O.ball_mask(M, M // 2 - 4))
    idx = rng.choice(ball, size=64, replace=False)
    h = 1e-3
    fd, an = [], []
    with torch.no_grad():
        base = (0.5 * g["vol"]).clone()
        for j in idx:
            for unit in (1.0, 1j):
                vp = base.clone().view(-1)
                vm = base.clone().view(-1)
                vp[j] += h * unit
                vm[j] -= h * unit
                Lp = _loss64(slice_project(vp.view(M, M, M), g["rot"], g["df"], geom), g["images"])
                Lm = _loss64(slice_project(vm.view(M, M, M), g["rot"], g["df"], geom), g["images"])
                fd.append((Lp - Lm) / (2 * h))
                gj = complex(grad.view(-1)[j].item())
                an.append(gj.real if unit == 1.0 else gj.imag)
    fd, an = np.array(fd), np.array(an)
    # FP32 forward values: each finite difference is accurate to ~1e-4 of the
    # gradient scale
    assert np.max(np.abs(fd - an)) <= 2e-3 * np.max(np.abs(an))


def test_gradcheck_small_double_path(dev):
    """torch.autograd.gradcheck-style check of the vector-Jacobian product:
    <J^T u, e> = <u, J e> for random u and e (the adjoint identity through
    autograd)."""
    from paper_2311_16100_gb300.autograd import slice_project
    c = Case(24, 7, interp="trilinear", ctf=True, seed=77)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    gen = torch.Generator(device="cuda").manual_seed(1)
    e = torch.randn((24, 24, 24), dtype=torch.complex64, device="cuda", generator=gen)
    u = torch.randn((7, 24, 24), dtype=torch.complex64, device="cuda", generator=gen)
    v = torch.zeros_like(e).requires_grad_(True)
    y = slice_project(v, g["rot"], g["df"], geom)
    (vjp,) = torch.autograd.grad(y, v, grad_outputs=u)
    Je = slice_project(e, g["rot"], g["df"], geom)
    lhs = torch.sum((torch.conj(vjp) * e).real.double())
    rhs = torch.sum((torch.conj(u) * Je).real.double())
    assert abs(float(lhs - rhs)) <= 1e-5 * abs(float(rhs))
