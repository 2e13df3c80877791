"""The ground truth v* of the time-to-error runs against the paper's solver.

bench.py computes v* = H^{-1} b on the GPU by conjugate gradients through the
library's gradient (reading 13: the paper's Section 4 uses L-BFGS; both reach
the minimiser of Eq. optim cp since H is SPD for lambda > 0).  Here that GPU
solve is compared with the FP64 oracle's L-BFGS on the same inputs (16^3,
120 images, trilinear, CTF)."""
import os
import sys

import numpy as np
import pytest

import oracle as O
from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_cg_ground_truth_matches_oracle_lbfgs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    import bench
    from paper_2311_16100_gb300 import ops, synth
    M, N, lam = 16, 120, 0.05
    c = Case(M, N, interp="trilinear", ctf=True, seed=161)
    g = c.to_gpu()
    h = ops.Handle(0)
    W = dict(geom=c.gpu_geometry(), images=g["images"], quat=g["quat"], df=g["df"], ctf=True)
    cfg = dict(M=M, interp="trilinear")
    vstar, _ = bench.ground_truth(h, torch, synth, W, cfg, lam)
    b = O.full_rhs(c.images, c.R, c.df, **c.geo())
    vl, it = O.lbfgs_solve(b, c.R, c.df, lam=lam, max_iter=1000, tol=1e-10, **c.geo())
    ball = O.ball_mask(M, c.r_max).reshape(M, M, M)
    vl = np.where(ball, vl, 0)
    assert it < 1000
    assert rel_l2(vstar.cpu().numpy(), vl) <= 1e-4
    h.close()
