"""Seeded synthetic inputs shaped like the paper's refinement workloads.

This module only draws random inputs: Fourier volumes built from Gaussian
blobs, uniformly distributed rotations (as unit quaternions), per-image
defocus values, the epoch permutation and an initial iterate.  It holds none
of the reconstruction method's arithmetic (no projection, no CTF, no loss), so
it can feed both the CUDA path and the CPU oracle.

Conventions shared by every caller (Section 2.1 of the paper leaves the
ordering open, "without loss of generality"):

* grid side ``M`` is even; voxel ``(iz, iy, ix)`` has linear index
  ``(iz*M + iy)*M + ix`` and frequency coordinates
  ``(kx, ky, kz) = (ix - M/2, iy - M/2, iz - M/2)`` (DC at index ``M/2``);
* a volume is ``complex64[M][M][M]``; an image is ``complex64[M][M]`` indexed
  ``[iy][ix]``;
* quaternions are ``(w, x, y, z)``, Hamilton convention, unit norm.
"""
from __future__ import annotations

import numpy as np

# Microscope constants of the synthetic workloads (300 kV, Cs 2.7 mm,
# amplitude contrast 0.1, pixel 1.5 A).
CTF_KV = 300.0
CTF_CS_MM = 2.7
CTF_AMP = 0.1
CTF_PIXEL_A = 1.5

# Blob count per grid side: 20 / 200 / 1000 / 5000 blobs for M = 32/64/128/256.
BLOBS_FOR_M = {32: 20, 64: 200, 128: 1000, 256: 5000}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def blob_volume(M: int, n_blobs: int | None = None, sigma: float = 1.5,
                seed: int = 0) -> np.ndarray:
    """Fourier volume of ``n_blobs`` Gaussian blobs (centred convention).

    Blobs of width ``sigma`` voxels sit uniformly inside the ball of radius
    M/4 about the box centre with amplitudes U[0.5, 1.5].  The real-space
    volume is rendered locally around each blob, transformed with a 3-D DFT
    whose origin is the box centre, and shifted so that DC sits at index M/2.
    The result is scaled so that the mean |v|^2 over the ball of radius
    M/2-1 is 1.  Returns complex64[M][M][M].
    """
    if n_blobs is None:
        n_blobs = BLOBS_FOR_M.get(M, max(4, M // 2))
    g = rng(seed)
    # uniform in a ball: radius ~ R u^(1/3), direction isotropic
    d = g.normal(size=(n_blobs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = (M / 4.0) * g.random(n_blobs) ** (1.0 / 3.0)
    centres = M / 2.0 + d * r[:, None]          # (x, y, z) in voxel units
    amps = g.uniform(0.5, 1.5, size=n_blobs)
    real = np.zeros((M, M, M), dtype=np.float64)   # [z][y][x]
    half = int(np.ceil(5 * sigma))
    ax = np.arange(-half, half + 1)
    for c, a in zip(centres, amps):
        ic = np.floor(c).astype(int)
        ix = ic[0] + ax
        iy = ic[1] + ax
        iz = ic[2] + ax
        gx = np.exp(-0.5 * ((ix - c[0]) / sigma) ** 2)
        gy = np.exp(-0.5 * ((iy - c[1]) / sigma) ** 2)
        gz = np.exp(-0.5 * ((iz - c[2]) / sigma) ** 2)
        blk = a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        ok_x = (ix >= 0) & (ix < M)
        ok_y = (iy >= 0) & (iy < M)
        ok_z = (iz >= 0) & (iz < M)
        real[np.ix_(iz[ok_z], iy[ok_y], ix[ok_x])] += blk[np.ix_(ok_z, ok_y, ok_x)]
    vol = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(real)))
    q = ball_mask(M, M // 2 - 1)
    scale = np.sqrt(np.mean(np.abs(vol[q]) ** 2))
    return (vol / scale).astype(np.complex64)


def ball_mask(M: int, r_max: int) -> np.ndarray:
    """Boolean [M][M][M]: voxels with kx^2+ky^2+kz^2 <= r_max^2."""
    k = np.arange(M) - M // 2
    q = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    return q <= r_max * r_max


def shoemake_quaternions(n: int, seed: int) -> np.ndarray:
    """n uniformly distributed unit quaternions (w, x, y, z), float64.

    Shoemake's subgroup algorithm (K. Shoemake, "Uniform random rotations",
    Graphics Gems III, 1992): from u1, u2, u3 ~ U[0,1),
    q = (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2,
         sqrt(u1) sin 2pi u3, sqrt(u1) cos 2pi u3).
    """
    g = rng(seed)
    u = g.random((n, 3))
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2 * np.pi * u[:, 1]
    t2 = 2 * np.pi * u[:, 2]
    q = np.stack([a * np.sin(t1), a * np.cos(t1), b * np.sin(t2), b * np.cos(t2)], axis=1)
    # canonical sign (w >= 0); q and -q are the same rotation
    q[q[:, 0] < 0] *= -1
    return q


def defocus_angstrom(n: int, seed: int, lo_um: float = 1.0, hi_um: float = 3.0) -> np.ndarray:
    """Per-image defocus in Angstrom, U[lo, hi] micrometres, float64."""
    return rng(seed).uniform(lo_um * 1e4, hi_um * 1e4, size=n)


def complex_normal(shape, seed: int, var: float = 1.0) -> np.ndarray:
    """Circular complex Gaussian with E|z|^2 = var (re, im ~ N(0, var/2))."""
    g = rng(seed)
    s = np.sqrt(var / 2.0)
    return s * g.normal(size=shape) + 1j * s * g.normal(size=shape)


def initial_volume(M: int, r_max: int, tau2: float, seed: int) -> np.ndarray:
    """Random starting iterate: CN(0, tau2) inside the ball, 0 outside."""
    v = complex_normal((M, M, M), seed, tau2)
    v[~ball_mask(M, r_max)] = 0
    return v.astype(np.complex64)


def permutation(n: int, seed: int) -> np.ndarray:
    return rng(seed).permutation(n)


def config_seed(config_index: int, dataset_index: int = 0) -> int:
    """Seed rule of the synthetic workloads: config index * 1000 + dataset."""
    return 1000 * config_index + dataset_index
