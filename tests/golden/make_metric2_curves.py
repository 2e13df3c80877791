"""Write the oracle's relative-error curves of the 32^3 refinement workload.

Workload (the smallest of the paper-shaped synthetic workloads): a 32^3
Fourier volume of 20 Gaussian blobs, 1000 images with uniform random
rotations, nearest interpolation, no CTF, complex Gaussian noise at SNR 0.1,
lambda = sigma^2 / tau^2 with tau^2 = 1, Algorithm 1 with batch 100 for 5
epochs (50 iterations, 16 probes per Hutchinson estimate), beta = 0.9,
c = 0.5, eta^0 = 1, alpha of Eq. thresh value over the whole dataset.
Three arms from the same start and the same per-epoch permutations:
  plain        D-hat = I (stochastic Armijo gradient descent);
  hutchinson   Algorithm 1 (Eqs. hutch update, exp avg update, thresh);
  precomputed  a fixed D from Eq. diag est rule over the dataset (Section 4's
               precomputed arm; under nearest interpolation every estimate is
               exact, so one pass gives the same D as any number of passes).
After every iteration the relative error |v - v*| / |v*| over the ball,
v* = H^{-1} b the full-data minimiser (closed form under nearest
interpolation), is recorded with the accepted step size.

Besides, the same problem with the whole dataset as one batch (the
alternative reading of the batch that shows which ingredient sets the
mini-batch curves' floor): 10 iterations of each arm.

Everything here calls only the oracle and the seeded input generator.
Run:  python tests/golden/make_metric2_curves.py  (about a minute)
writes tests/golden/metric2_m32_curves.txt.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2311_16100_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "metric2_m32_curves.txt")
P = dict(M=32, n_img=1000, B=100, epochs=5, K=16, snr=0.1, blobs=20, seed=1000,
         beta=0.9, c=0.5, eta0=1.0)


def problem():
    """Inputs of the workload (seeded), the ground truth and the threshold."""
    M, N, seed = P["M"], P["n_img"], P["seed"]
    r = M // 2 - 1
    v_true = synth.blob_volume(M, P["blobs"], seed=seed)
    R = O.quat_to_rot(synth.shoemake_quaternions(N, seed + 1)).astype(np.float32)
    df = np.zeros(N, dtype=np.float32)
    clean = O.slice_project(v_true, R, df, M, r, "nearest", None)
    m = O.disc_mask(M, r).reshape(M, M)
    sig2 = float(np.mean(np.abs(clean[:, m]) ** 2) / P["snr"])
    noise = synth.complex_normal((N, M, M), seed + 3, sig2)
    noise[:, ~m] = 0
    x = (clean + noise).astype(np.complex64)
    lam = sig2
    b = O.full_rhs(x, R, df, M, r, "nearest", None)
    diag = O.exact_diag(R, df, M, r, "nearest", None, lam, 1.0)
    vstar = np.where(O.ball_mask(M, r).reshape(M, M, M), b / diag, 0)
    alpha = O.alpha_threshold(df, M, r, None, lam)
    v0 = synth.initial_volume(M, r, 1.0, seed + 7)
    perms = [synth.permutation(N, seed + 31 + ep) for ep in range(P["epochs"])]
    return dict(M=M, r=r, R=R, df=df, x=x, lam=lam, vstar=vstar, alpha=alpha, v0=v0,
                perms=perms)


def precomputed_D(S):
    return O.precomputed_preconditioner(S["R"], S["df"], S["M"], S["r"], "nearest", None,
                                        S["lam"], P["B"], 1, P["K"], P["seed"] + 13)


def run_arm(S, mode, D0, batch, epochs, perms):
    """Algorithm 1 for one arm; returns [(iteration, rel_err, eta)]."""
    M, r, N = S["M"], S["r"], len(S["R"])
    v = S["v0"].astype(np.complex128)
    D, Da, eta = (np.ones((M, M, M)) if D0 is None else D0), np.zeros((M, M, M)), P["eta0"]
    rows, k = [], 0
    for ep in range(epochs):
        perm = perms[ep] if perms is not None else np.arange(N)
        for s in range(0, N, batch):
            idx = perm[s:s + batch]
            k += 1
            out = O.alg1_step(v, D, Da, eta, k, S["x"][idx], S["R"][idx], S["df"][idx], M, r,
                              "nearest", None, S["lam"], N / len(idx), S["alpha"], P["beta"],
                              P["c"], mode, n_probes=P["K"], seed=P["seed"] + 11)
            v, D, Da, eta = out["v"], out["D"], out["D_avg"], out["eta"]
            rows.append((k, O.rel_err(v, S["vstar"], M, r), eta))
    return rows


ARMS = (("plain", "plain"), ("hutchinson", "hutchinson"), ("precomputed", "fixed"))


def main():
    S = problem()
    Dpre = precomputed_D(S)
    lines = ["# Oracle relative-error curves, 32^3 nearest, no CTF, 1000 images, SNR 0.1,",
             "# Algorithm 1 (Section 3.4) with the stochastic Armijo rule; written by",
             "# tests/golden/make_metric2_curves.py from the oracle only.",
             f"# lambda {S['lam']:.9g}  alpha {S['alpha']:.9g}",
             "# columns: setting arm iteration rel_err eta"]
    for setting, batch, epochs, perms in (("batch100", P["B"], P["epochs"], S["perms"]),
                                          ("fullbatch", P["n_img"], 10, None)):
        for arm, mode in ARMS:
            rows = run_arm(S, mode, Dpre if mode == "fixed" else None, batch, epochs, perms)
            for k, e, eta in rows:
                lines.append(f"{setting} {arm} {k} {e:.9e} {eta:.9g}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
