"""Learned diagonal preconditioner (not in the paper).

A 3 -> 64 -> 64 -> 1 network predicts log(diag(H) - lambda) per voxel from
features that cost one pose-only pass over the dataset (cs_exact_diag's
coverage and accumulated-CTF^2 outputs), so that preconditioned SGD can start
from a good D at iteration 1 instead of Algorithm 1's D^(0) = I.  It is
trained on Hutchinson estimates (Eq. hutch) that the method itself
generates; Hutchinson remains the fallback and the judge of its error.
Forward and gradient run in the library's BF16 tensor-core kernels; the
optimiser is the library's Adam step.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .ops import Geometry, Handle

# parameter layout of the library: W1[64][3] b1[64] W2[64][64] b2[64] w3[64] b3
SIZES = (("W1", 192), ("b1", 64), ("W2", 4096), ("b2", 64), ("w3", 64), ("b3", 1))


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation, float32 [4481]."""
    g = np.random.Generator(np.random.PCG64(seed))
    fan = {"W1": 3, "b1": 3, "W2": 64, "b2": 64, "w3": 64, "b3": 64}
    parts = [g.uniform(-1 / math.sqrt(fan[n]), 1 / math.sqrt(fan[n]), size=k) for n, k in SIZES]
    return np.concatenate(parts).astype(np.float32)


class Sample:
    """Features and target of one dataset (all on the device)."""

    def __init__(self, M, r_ball, coverage, ctf2w, target):
        self.M, self.r_ball = M, r_ball
        self.coverage, self.ctf2w, self.target = coverage, ctf2w, target


def dataset_features(h: Handle, geom: Geometry, rot, defocus, subsample: int = 1):
    """(coverage, sum C^2 w) per voxel, estimated for the whole dataset of N
    poses from its first ceil(N / subsample) poses (one pose-only pass over
    them, scaled by N / their number; subsample = 1: the exact sums)."""
    N = rot.shape[0]
    n = -(-N // subsample)
    _, cov, c2w = h.exact_diag(geom, rot[:n], defocus[:n] if defocus is not None else None,
                               0.0, N / n, diag=False, coverage=True, ctf2w=True)
    return cov, c2w


def hutchinson_target(h: Handle, geom: Geometry, rot, defocus, n_probes=32, n_blocks=4,
                      seed=12345, floor=1e-3):
    """log(max(D_hutch, floor * mean)) with D_hutch the Hutchinson estimate of
    diag(sum_i P_i^* C_i^2 P_i) over the dataset (lambda = 0), averaged over
    n_blocks independent probe blocks of n_probes probes (cs_mlp_target)."""
    M = geom.M
    est = torch.empty((n_blocks, M, M, M), dtype=torch.float32, device=rot.device)
    for blk in range(n_blocks):
        h.hutchinson_diag(geom, rot, defocus, 0.0, 1.0, n_probes=n_probes, seed=seed,
                          probe_block=blk + 1, out=est[blk])
    return h.mlp_target(M, est, floor)


class LearnedPreconditioner:
    def __init__(self, handle: Handle, seed: int = 0, tensor_cores: bool = True):
        self.h = handle
        self.tc = tensor_cores
        dev = torch.device("cuda", handle.device)
        self.params = torch.from_numpy(init_params(seed)).to(dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.sse = torch.zeros((), dtype=torch.float64, device=dev)
        self.step = 0

    def loss(self, samples) -> float:
        """Mean over samples of the per-sample mean squared error."""
        tot = 0.0
        for s in samples:
            self.sse.zero_()
            g = torch.zeros_like(self.grad)
            self.h.mlp_grad(s.M, s.r_ball, self.params, s.coverage, s.ctf2w, s.target, g,
                            self.sse, self.tc)
            tot += float(self.sse) / s.n_ball
        return tot / len(samples)

    def fit(self, samples, steps=300, lr=1e-2):
        """Full-batch Adam over all samples; returns the loss history."""
        for s in samples:
            s.n_ball = int(torch.count_nonzero(_ball(s.M, s.r_ball, self.params.device)))
        hist = []
        for _ in range(steps):
            self.sse.zero_()
            for s in samples:
                # each sample's mean squared error, averaged over samples
                self.h.mlp_grad(s.M, s.r_ball, self.params, s.coverage, s.ctf2w, s.target,
                                self.grad, self.sse, self.tc)
            self.step += 1
            self.h.mlp_adam_step(self.params, self.m, self.v, self.grad, self.step, lr,
                                 grad_scale=1.0 / len(samples))
            hist.append(float(self.sse))
        self.h.check_device_status()
        return hist

    def predict(self, M, coverage, ctf2w, lam=0.0):
        """Predicted preconditioner D = exp(network) + lambda, float32 [M][M][M]."""
        return self.h.mlp_forward(M, self.params, coverage, ctf2w, exp=True, offset=lam,
                                  tensor_cores=self.tc)


def _ball(M, r, device):
    k = torch.arange(M, device=device) - M // 2
    q = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    return q <= r * r
