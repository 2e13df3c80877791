"""Oracle: Rademacher probes and Hutchinson's diagonal estimator (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from .operators import _image_terms, hvp

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MASK32 = np.uint64(0xFFFFFFFF)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output number ``c`` (0-based) of a SplitMix64 stream seeded with ``seed``.

    SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
    number generators", OOPSLA 2014; finaliser constants of S. Vigna's public
    reference code): state_c = seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64),
    z = (s ^ s>>30) * 0xBF58476D1CE4E5B9, z = (z ^ z>>27) * 0x94D049BB133111EB,
    output z ^ z>>31.  Counter based, so any output is drawn directly.
    """
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(seed) + (c + np.uint64(1)) * GOLDEN_GAMMA
        z = (s ^ (s >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def probe_words(seed: int, block: int, n_vox: int) -> np.ndarray:
    """32 probe bits per voxel for probe block ``block``: uint32 [n_vox].

    Voxels are taken in pairs (2i, 2i+1): both words come from SplitMix64
    output number block*ceil(n_vox/2) + i, the low 32 bits for voxel 2i and
    the high 32 bits for voxel 2i+1.
    """
    n_pairs = (n_vox + 1) // 2
    j = np.arange(n_vox, dtype=np.uint64)
    c = np.uint64(block) * np.uint64(n_pairs) + (j >> np.uint64(1))
    out = splitmix64(seed, c)
    half = (j & np.uint64(1)) * np.uint64(32)
    return ((out >> half) & _MASK32).astype(np.uint32)


def rademacher_probes(seed: int, block: int, n_vox: int, n_probes: int) -> np.ndarray:
    """Rademacher(0.5) vectors z_k, k < n_probes <= 32 (Eq. hutch): [K][n_vox].

    z_kj = +1 if bit k of voxel j's probe word is 0, -1 if it is 1.
    """
    if not 1 <= n_probes <= 32:
        raise ValueError("n_probes must be in 1..32")
    w = probe_words(seed, block, n_vox).astype(np.int64)
    bits = (w[None, :] >> np.arange(n_probes)[:, None]) & 1
    return 1.0 - 2.0 * bits


def hutchinson_diag(R, defocus, M, r_max, interp, ctf, lam, scale,
                    n_probes, seed, block):
    """D_est = (1/K) sum_k z_k (.) H_I z_k  (Eq. hutch, K probes, Section 3.2).

    Computed literally: K Hessian-vector products with the mini-batch
    Hessian, each multiplied element-wise by its probe, then averaged.
    """
    n = M ** 3
    Z = rademacher_probes(seed, block, n, n_probes)
    acc = np.zeros(n)
    for k in range(n_probes):
        acc += Z[k] * hvp(Z[k], R, defocus, M, r_max, interp, ctf, lam, scale).ravel()
    return (acc / n_probes).reshape(M, M, M)


def hutchinson_diag_at(voxels, R, defocus, M, r_max, interp, ctf, lam, scale,
                       n_probes, seed, block):
    """Entries ``voxels`` of hutchinson_diag (Eq. hutch, same probes),
    computed literally for those rows only, for checking a full-size
    estimate at sampled voxels:

        D_j = (1/K) sum_k z_kj (H_I z_k)_j,
        (H_I z)_j = lam z_j + scale sum_i sum_p C_ip^2 w_pj (P_i z)_p,

    the inner sum running over the pixels p whose interpolation stencil
    holds voxel j.  Since z_kj^2 = 1 the lam term is lam.  Returns float64
    [len(voxels)]."""
    vox_sel = np.asarray(voxels, dtype=np.int64)
    if len(np.unique(vox_sel)) != len(vox_sel):
        raise ValueError("voxels must be distinct")
    n = M ** 3
    words = probe_words(seed, block, n).astype(np.int64)
    ks = np.arange(n_probes)
    acc = np.zeros(len(vox_sel))
    order = np.argsort(vox_sel)
    sorted_sel = vox_sel[order]
    for i in range(len(R)):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        hit = np.isin(vox, sorted_sel) & (w != 0)
        rows = np.nonzero(hit.any(axis=1))[0]
        for p in rows:
            z = 1.0 - 2.0 * ((words[vox[p]][None, :] >> ks[:, None]) & 1)   # [K][c]
            pz = z @ w[p]                                                  # (P_i z_k)_p
            for c in np.nonzero(hit[p])[0]:
                j = order[np.searchsorted(sorted_sel, vox[p, c])]
                acc[j] += C[p] ** 2 * w[p, c] * float(np.dot(z[:, c], pz)) / n_probes
    return lam + scale * acc
