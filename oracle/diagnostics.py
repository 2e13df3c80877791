"""Oracle: convergence and conditioning diagnostics (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Fourier shell correlation (Eq. fsc, Section 4) between two volumes over
  1-voxel shells S_r = {k : round(|k|) = r}.
* Per-shell minimum / maximum of a real field, and from them the condition
  number of diag(H) restricted to the ball of radius R (Section 3.1: with
  nearest interpolation H is diagonal, so its condition number over the
  voxels |k| <= R is max H_jj / min H_jj there).
* The lower bound of Eq. cond number p, (N + lam) / (p(R) N + lam), with p(R)
  the ratio of pixels in the disc of radius R to voxels in the ball of
  radius R, both counted on the grid.
"""
from __future__ import annotations

import numpy as np


def shell_index(M: int) -> np.ndarray:
    """round(|k|) per voxel (z, y, x order), k = index - M/2; |k| is never a
    half-integer (|k|^2 is an integer), so the rounding has no ties."""
    k = np.arange(M) - M // 2
    q = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    return np.rint(np.sqrt(q.astype(np.float64))).astype(np.int64)


def fsc(u, v, M: int, n_shells: int):
    """(fsc[r], sums[r] = (Re sum u conj v, sum |u|^2, sum |v|^2)) for r < n_shells."""
    s = shell_index(M).ravel()
    u = np.asarray(u, np.complex128).ravel()
    v = np.asarray(v, np.complex128).ravel()
    sums = np.zeros((n_shells, 3))
    for r in range(n_shells):
        m = s == r
        sums[r, 0] = np.sum(u[m] * np.conj(v[m])).real
        sums[r, 1] = np.sum(np.abs(u[m]) ** 2)
        sums[r, 2] = np.sum(np.abs(v[m]) ** 2)
    den = sums[:, 1] * sums[:, 2]
    out = np.zeros(n_shells)
    ok = den > 0
    out[ok] = sums[ok, 0] / np.sqrt(den[ok])
    return out, sums


def shell_minmax(x, M: int, n_shells: int):
    """(min, max, count) of a real field per shell; +inf / -inf when empty."""
    s = shell_index(M).ravel()
    x = np.asarray(x, np.float64).ravel()
    lo = np.full(n_shells, np.inf)
    hi = np.full(n_shells, -np.inf)
    cnt = np.zeros(n_shells, np.int64)
    for r in range(n_shells):
        m = s == r
        cnt[r] = m.sum()
        if cnt[r]:
            lo[r] = x[m].min()
            hi[r] = x[m].max()
    return lo, hi, cnt


def condition_by_radius(diag, M: int, radii):
    """kappa(R) = max / min of diag over the ball round(|k|) <= R."""
    s = shell_index(M)
    d = np.asarray(diag, np.float64)
    return np.array([d[s <= R].max() / d[s <= R].min() for R in radii])


def p_ratio(M: int, R: int) -> float:
    """Pixels in the disc round(|k|) <= R over voxels in the ball round(|k|) <= R."""
    k = np.arange(M) - M // 2
    q2 = k[:, None] ** 2 + k[None, :] ** 2
    n2 = int(np.sum(np.rint(np.sqrt(q2)) <= R))
    n3 = int(np.sum(shell_index(M) <= R))
    return n2 / n3


def kappa_lower_bound(N: int, lam: float, p: float) -> float:
    """Eq. cond number p: (N + lam) / (p N + lam), valid when 1/p <= N."""
    return (N + lam) / (p * N + lam)
