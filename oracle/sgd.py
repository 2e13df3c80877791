"""Oracle: threshold alpha, Algorithm 1, ground truth and error (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from .geometry import ball_mask, ctf_pixels
from .hutchinson import hutchinson_diag
from .operators import backproject_adjoint, hvp, loss, loss_grad


def shell_counts(M: int, R: int):
    """(P_x(R), P_v(R)): pixels / voxels of the grid in the Fourier shell R.

    Section 3.3 leaves the shell width open; we take 1-voxel shells,
    round(|k|) = R, i.e. R^2 - R + 1 <= |k|^2 <= R^2 + R for integer R >= 1
    (|k|^2 is an integer, so no point sits on a half-integer radius).
    """
    k = np.arange(M) - M // 2
    lo, hi = R * R - R + 1, R * R + R
    q2 = k[:, None] ** 2 + k[None, :] ** 2
    q3 = q2[None, :, :] + (k ** 2)[:, None, None]
    return int(np.count_nonzero((q2 >= lo) & (q2 <= hi))), \
        int(np.count_nonzero((q3 >= lo) & (q3 <= hi)))


def alpha_threshold(defocus_all, M, r_max, ctf, lam, scale_alpha=1.0, R=None):
    """alpha = H-bar of Eq. (thresh value), at the maximum radius R = r_max.

    H-bar = P_x(R)/P_v(R) * sum_{i=1}^N |C_i(R)|^2 + lam, the expected Hessian
    entry at radius R for uniform orientations; C_i(R) is the CTF of image i
    at |k| = R (ones without CTF).  ``scale_alpha`` multiplies the sum (1 when
    ``defocus_all`` holds the whole dataset).  ``R`` overrides the radius.
    """
    if R is None:
        R = r_max
    Px, Pv = shell_counts(M, R)
    d = np.asarray(defocus_all, dtype=np.float64)
    if ctf is None:
        c2 = float(d.size)
    else:
        c2 = sum(float(ctf_pixels(float(R * R), di, M, ctf)) ** 2 for di in d)
    return Px / Pv * scale_alpha * float(c2) + lam


def alg1_step(v, D, D_avg, eta_prev, k, images, R, defocus, M, r_max, interp,
              ctf, lam, scale, alpha, beta, c, mode, n_probes=1, seed=0,
              max_halvings=64):
    """One iteration k (1-based) of Algorithm 1, executed literally.

    mode "hutchinson": Hutchinson's estimate on the batch with fresh probes
    (probe block k), running mean D_avg (Eq. hutch update as written in the
    algorithm), EMA D (Eq. exp avg update), threshold (Eq. thresh).
    mode "fixed": D is given (a precomputed preconditioner), thresholded.
    mode "plain": no preconditioner (D-hat = I).
    Then eta = eta_prev, v+ = v - eta D-hat^{-1} g, halving eta while the
    stochastic Armijo condition (Eq. stochastic armijo) fails, with f_I
    re-evaluated at every trial point.
    Returns dict(v, D, D_avg, eta, halvings, loss, G).
    """
    v = np.asarray(v, dtype=np.complex128)
    if mode == "hutchinson":
        D_est = hutchinson_diag(R, defocus, M, r_max, interp, ctf, lam, scale,
                                n_probes, seed, k)
        D_avg = (k - 1) / k * D_avg + D_est / k
        D = beta * D + (1 - beta) * D_avg
        Dhat = np.maximum(np.abs(D), alpha)
    elif mode == "fixed":
        Dhat = np.maximum(np.abs(D), alpha)
    elif mode == "plain":
        Dhat = np.ones((M, M, M))
    else:
        raise ValueError(mode)
    f0, g = loss_grad(v, images, R, defocus, M, r_max, interp, ctf, lam, scale)
    d = g / Dhat
    G = float(np.sum(np.abs(g) ** 2 / Dhat))
    eta = eta_prev
    v_new = v - eta * d
    h = 0
    while (loss(v_new, images, R, defocus, M, r_max, interp, ctf, lam, scale)
           > f0 - c * eta * G) and h < max_halvings:
        eta /= 2
        v_new = v - eta * d
        h += 1
    return dict(v=v_new, D=D, D_avg=D_avg, eta=eta, halvings=h, loss=f0, G=G)


def precomputed_preconditioner(R_all, defocus_all, M, r_max, interp, ctf, lam, B, n_epochs,
                               n_probes, seed):
    """The preconditioner estimated in advance (Section 4's precomputed arm):
    Eq. diag est rule run over n_epochs passes of the dataset in batches of B
    (the last batch may be short), each batch's Hutchinson estimate taken with
    its own scale N/|I| (Eq. optim cp's batch reading) and probe block k = the
    running iteration count, and averaged with the running mean
    D = ((k-1)/k) D + (1/k) est.  Images are taken in the given order."""
    N = R_all.shape[0]
    D = np.zeros((M, M, M))
    k = 0
    for _ in range(n_epochs):
        for start in range(0, N, B):
            sl = slice(start, min(start + B, N))
            nb = sl.stop - sl.start
            k += 1
            df = np.zeros(nb) if defocus_all is None else defocus_all[sl]
            est = hutchinson_diag(R_all[sl], df, M, r_max, interp, ctf, lam, N / nb,
                                  n_probes, seed, k)
            D = ((k - 1) / k) * D + (1.0 / k) * est
    return D


def full_rhs(images, R, defocus, M, r_max, interp, ctf):
    """b = sum_i P_i^* C_i x_i over the whole dataset (Eq. lin sys)."""
    return backproject_adjoint(images, R, defocus, M, r_max, interp, ctf)


def cg_solve(b, R, defocus, M, r_max, interp, ctf, lam, tol=1e-12, max_iter=2000):
    """v* solving H v = b (Eq. lin sys), by conjugate gradients in FP64.

    The paper computes its ground truth with L-BFGS; for lam > 0 H is SPD and
    CG on H v = b reaches the same minimiser.  H is real, so the real and
    imaginary parts are two independent systems solved together.
    """
    def Hmul(x):
        return (hvp(x.real, R, defocus, M, r_max, interp, ctf, lam, 1.0)
                + 1j * hvp(x.imag, R, defocus, M, r_max, interp, ctf, lam, 1.0))
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.sqrt(np.vdot(b, b).real)
    for it in range(max_iter):
        if np.sqrt(rr) <= tol * bn:
            break
        Hp = Hmul(p)
        a = rr / np.vdot(p, Hp).real
        x += a * p
        r -= a * Hp
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, it


def lbfgs_solve(b, R, defocus, M, r_max, interp, ctf, lam, memory=10, max_iter=1000,
                tol=1e-12):
    """v* minimising Eq. (optim cp), f(v) = 1/2 <v, H v> - <b, v> + const, by
    L-BFGS (Liu & Nocedal 1989), the paper's ground-truth solver (Section 4,
    1000 iterations there).

    The search direction comes from the two-loop recursion over the last
    ``memory`` pairs s = v_{k+1} - v_k, y = g_{k+1} - g_k, with the initial
    scaling gamma = <s, y> / <y, y>; since f is quadratic the step length is
    the exact minimiser along the direction, t = -<g, p> / <p, H p>.  Complex
    volumes are real vectors of twice the length (H acts alike on the real
    and imaginary parts).  Stops when |g| <= tol |b| or after max_iter
    iterations.  Returns (v, iterations)."""
    def Hmul(x):
        return (hvp(x.real, R, defocus, M, r_max, interp, ctf, lam, 1.0)
                + 1j * hvp(x.imag, R, defocus, M, r_max, interp, ctf, lam, 1.0))

    def dot(a, c):
        return float(np.vdot(a, c).real)

    b = np.asarray(b, dtype=np.complex128)
    v = np.zeros_like(b)
    g = -b                                  # gradient H v - b at v = 0
    bn = np.sqrt(dot(b, b))
    S, Y = [], []
    it = 0
    for it in range(max_iter):
        if np.sqrt(dot(g, g)) <= tol * bn:
            break
        q = g.copy()
        alphas = []
        for s_i, y_i in zip(reversed(S), reversed(Y)):
            a_i = dot(s_i, q) / dot(y_i, s_i)
            alphas.append(a_i)
            q = q - a_i * y_i
        if S:
            q = q * (dot(S[-1], Y[-1]) / dot(Y[-1], Y[-1]))
        for (s_i, y_i), a_i in zip(zip(S, Y), reversed(alphas)):
            beta = dot(y_i, q) / dot(y_i, s_i)
            q = q + (a_i - beta) * s_i
        p = -q
        Hp = Hmul(p)
        t = -dot(g, p) / dot(p, Hp)
        s_new = t * p
        y_new = t * Hp                       # g_{k+1} - g_k = H s
        v = v + s_new
        g = g + y_new
        S.append(s_new)
        Y.append(y_new)
        if len(S) > memory:
            S.pop(0)
            Y.pop(0)
    return v, it


def rel_err(v, v_star, M, r_max):
    """|v - v*| / |v*| over the ball |k| <= r_max (voxels outside are unseen)."""
    m = ball_mask(M, r_max)
    a = np.asarray(v).ravel()[m]
    b = np.asarray(v_star).ravel()[m]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
