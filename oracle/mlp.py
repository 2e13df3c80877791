"""Oracle: the learned diagonal preconditioner's network (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Not in the paper: a
3 -> 64 -> 64 -> 1 multilayer perceptron with GELU activations maps per-voxel
features (radial frequency, pose coverage, accumulated CTF^2) to log D, the
logarithm of the diagonal preconditioner; it is trained by mean squared
error against Hutchinson estimates (Eq. hutch) of the diagonal.

The GPU runs the 64 x 64 layer on BF16 tensor cores with FP32 accumulation:
its operands (the first hidden activations and the layer's weights) are
rounded to BF16, and so is the backward operand (the gradient at the second
hidden layer).  This oracle computes everything in FP64 except for those
three roundings, which it applies at the same points.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
N_FEAT = 3


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rnd = ((u >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)
    u = ((u + rnd) >> np.uint64(16)) << np.uint64(16)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    """GELU with the tanh approximation (Hendrycks & Gimpel 2016):
    0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    c = math.sqrt(2.0 / math.pi)
    return 0.5 * x * (1.0 + np.tanh(c * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    c = math.sqrt(2.0 / math.pi)
    u = c * (x + 0.044715 * x ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * c * (1.0 + 3 * 0.044715 * x * x)


def features(M, coverage, ctf2w, idx=None):
    """Per-voxel features [M^3][3]: |k| / (M/2), log1p(coverage), log1p(sum C^2 w);
    with idx, only the voxels of those linear indices (z-major: j = (z M + y) M + x)."""
    if idx is None:
        k = np.arange(M) - M // 2
        kr = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
        kr = kr.ravel()
        cov = np.asarray(coverage, np.float64).ravel()
        c2w = np.asarray(ctf2w, np.float64).ravel()
    else:
        j = np.asarray(idx, np.int64)
        kx = j % M - M // 2
        ky = (j // M) % M - M // 2
        kz = j // (M * M) - M // 2
        kr = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
        cov = np.asarray(coverage).ravel()[j].astype(np.float64)
        c2w = np.asarray(ctf2w).ravel()[j].astype(np.float64)
    return np.stack([kr / (M / 2), np.log1p(cov), np.log1p(c2w)], axis=1)


def init_params(seed):
    """Deterministic initial parameters (uniform fan-in scaling)."""
    g = np.random.Generator(np.random.PCG64(seed))
    def u(shape, fan_in):
        b = 1.0 / math.sqrt(fan_in)
        return g.uniform(-b, b, size=shape)
    return dict(W1=u((H, N_FEAT), N_FEAT), b1=u((H,), N_FEAT), W2=u((H, H), H), b2=u((H,), H),
                w3=u((H,), H), b3=u((1,), H))


def forward(p, X, rounding=True):
    """y [n] = w3 . GELU(W2 bf(GELU(W1 x + b1)) + b2) + b3 with BF16 W2 and H1
    (rounding=False: the plain FP64 network)."""
    rd = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    A1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(A1)
    A2 = rd(H1) @ rd(p["W2"]).T + p["b2"]
    H2 = gelu(A2)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, dict(A1=A1, H1=H1, A2=A2, H2=H2)


def loss_and_grads(p, X, t, rounding=True):
    """Mean squared error L = mean (y - t)^2 and its parameter gradients.

    Backward through the 64 x 64 layer uses the BF16-rounded gradient dA2 and
    weights W2, as the tensor-core kernels do (rounding=False: the exact
    gradient of the plain FP64 network)."""
    rd = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    n = X.shape[0]
    y, c = forward(p, X, rounding)
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = c["H2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dA2 = (dy[:, None] * p["w3"][None, :]) * gelu_grad(c["A2"])
    dA2b = rd(dA2)
    g["W2"] = dA2b.T @ rd(c["H1"])
    g["b2"] = dA2.sum(axis=0)
    dH1 = dA2b @ rd(p["W2"])
    dA1 = dH1 * gelu_grad(c["A1"])
    g["W1"] = dA1.T @ X
    g["b1"] = dA1.sum(axis=0)
    return L, g
