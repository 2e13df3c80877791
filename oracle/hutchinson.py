"""Oracle: Rademacher probes and Hutchinson's diagonal estimator (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from .operators import hvp

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
