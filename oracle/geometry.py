"""Oracle: grid, rotations, interpolation stencils and the CTF (FP64, CPU).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package;
only the tests, the smoke check and the CPU-baseline leg of the benchmark do.

Every function follows a passage of Toader, Brubaker & Lederman,
"Efficient high-resolution refinement in cryo-EM with stochastic gradient
descent" (arXiv 2311.16100), cited in its docstring.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------- grid
def freq_axis(M: int) -> np.ndarray:
    """Frequency coordinate of each index along one axis: k = i - M/2.

    Section 2.1 fixes only that the image grid is the z=0 plane of the volume
    grid; the centred ordering is our (equivalent) relabelling.
    """
    return np.arange(M) - M // 2


def pixel_coords(M: int):
    """(kx, ky) of every pixel of an M x M image, flattened [iy][ix]."""
    k = freq_axis(M)
    ky, kx = np.meshgrid(k, k, indexing="ij")
    return kx.ravel(), ky.ravel()


def shift_phase(M: int, shifts) -> np.ndarray:
    """In-plane shift operators of Definition 2.1 as phases [B][M][M]:
    T_i(k) = exp(-2 pi i (kx tx_i + ky ty_i) / M) for shifts (tx, ty) in
    pixels (the paper gives no formula; this is the Fourier shift theorem for
    a real-space shift by +t)."""
    kx, ky = pixel_coords(M)
    t = np.asarray(shifts, np.float64).reshape(-1, 2)
    a = (kx[None, :] * t[:, :1] + ky[None, :] * t[:, 1:]) / M
    return np.exp(-2j * np.pi * a).reshape(-1, M, M)


def phase_shift(images, shifts, sign=-1):
    """images * T (sign +1) or images * conj(T) (sign -1)."""
    M = images.shape[-1]
    T = shift_phase(M, shifts)
    return np.asarray(images, np.complex128) * (T if sign > 0 else np.conj(T))


def disc_mask(M: int, r_max: int) -> np.ndarray:
    """Pixels used by the model: kx^2 + ky^2 <= r_max^2 (flattened)."""
    kx, ky = pixel_coords(M)
    return kx * kx + ky * ky <= r_max * r_max


def ball_mask(M: int, r_max: int) -> np.ndarray:
    """Voxels with |k| <= r_max, flattened (z, y, x) order."""
    k = freq_axis(M)
    q = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    return (q <= r_max * r_max).ravel()


def default_r_max(M: int) -> int:
    return M // 2 - 1


# ---------------------------------------------------------------- rotations
def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Unit quaternion(s) (w, x, y, z) -> rotation matrix R (row-major 3x3).

    The pose of Definition 2.1 carries a rotation matrix R in SO(3); the paper
    does not say how R is parameterised.  Quaternions use the Hamilton
    convention: R v equals the vector part of q (0, v) q*.  The quaternion is
    normalised first.
    """
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def sample_points(R: np.ndarray, kx: np.ndarray, ky: np.ndarray) -> np.ndarray:
    """Points R^T r of the volume read by pixels r = (kx, ky, 0), FP64.

    Section 2.1: (R v)(r) = v(R^T r), so pixel r of the projection reads the
    volume at R^T r.  Component a is R[0][a] kx + R[1][a] ky.  Returns [n, 3]
    as (x, y, z).
    """
    R = np.asarray(R, dtype=np.float64)
    return kx[:, None] * R[0][None, :] + ky[:, None] * R[1][None, :]


def nearest_coords_fp32(R32: np.ndarray, kx: np.ndarray, ky: np.ndarray) -> np.ndarray:
    """Nearest grid point of R^T r, Eq. (def nn interp), in the FP32 reading.

    k*(j) = argmin_k |r_k - R^T r_j|; on a product grid this is the per-axis
    nearest integer.  The paper fixes neither the precision nor the tie rule;
    we read it as: each coordinate c_a = fl32(fl32(R[0][a]*kx) + fl32(R[1][a]*ky))
    (two single-precision products and one sum, no fused multiply-add),
    rounded half to even.  Returns int64 [n, 3] (x, y, z) frequency coords.
    """
    R32 = np.asarray(R32, dtype=np.float32)
    fx = kx.astype(np.float32)
    fy = ky.astype(np.float32)
    c = np.empty((kx.shape[0], 3), dtype=np.float32)
    for a in range(3):
        p0 = np.multiply(R32[0, a], fx, dtype=np.float32)
        p1 = np.multiply(R32[1, a], fy, dtype=np.float32)
        c[:, a] = np.add(p0, p1, dtype=np.float32)
    return np.rint(c).astype(np.int64)


def stencil(R32: np.ndarray, M: int, r_max: int, interp: str):
    """Rows of the projection matrix P_phi of Definition 2.1 for one image.

    Returns (pix, vox, w): ``pix`` [n] flat indices of the pixels inside the
    disc of radius r_max; ``vox`` [n, c] flat voxel indices and ``w`` [n, c]
    weights, with c = 1 (nearest, Eq. def nn interp) or c = 8 (trilinear,
    Eq. def tri interp).  A corner outside the grid gets weight 0 (and index
    0), so it contributes nothing either way.  No in-plane shift (T = I).
    """
    kx, ky = pixel_coords(M)
    m = kx * kx + ky * ky <= r_max * r_max
    pix = np.nonzero(m)[0]
    kx, ky = kx[m], ky[m]
    h = M // 2
    if interp == "nearest":
        n = nearest_coords_fp32(R32, kx, ky) + h          # grid indices
        ok = np.all((n >= 0) & (n < M), axis=1)
        vox = ((n[:, 2] * M + n[:, 1]) * M + n[:, 0])
        w = ok.astype(np.float64)
        vox = np.where(ok, vox, 0)
        return pix, vox[:, None], w[:, None]
    if interp != "trilinear":
        raise ValueError(interp)
    s = sample_points(np.asarray(R32, dtype=np.float64), kx, ky) + h
    i0 = np.floor(s).astype(np.int64)
    t = s - i0
    vox = np.empty((len(pix), 8), dtype=np.int64)
    w = np.empty((len(pix), 8))
    c = 0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix, iy, iz = i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz
                wx = t[:, 0] if dx else 1 - t[:, 0]
                wy = t[:, 1] if dy else 1 - t[:, 1]
                wz = t[:, 2] if dz else 1 - t[:, 2]
                ok = (ix >= 0) & (ix < M) & (iy >= 0) & (iy < M) & (iz >= 0) & (iz < M)
                vox[:, c] = np.where(ok, (iz * M + iy) * M + ix, 0)
                w[:, c] = np.where(ok, wx * wy * wz, 0.0)
                c += 1
    return pix, vox, w


# --------------------------------------------------------------------- CTF
def electron_wavelength_A(kv: float) -> float:
    """Relativistic electron wavelength in Angstrom for voltage kv (kV)."""
    V = kv * 1e3
    return 12.2643 / np.sqrt(V * (1.0 + 0.978466e-6 * V))


def ctf_of_s2(s2, defocus_A, kv, cs_mm, amp):
    """Weak-phase CTF at squared spatial frequency s2 (1/A^2).

    The paper only states that C_i is diagonal, real, radially symmetric and
    known with image-specific parameters (Sections 2.1, 3.3).  We use the
    textbook isotropic form without envelope:
      chi = pi lam df s^2 - (pi/2) Cs lam^3 s^4,
      C   = -(sqrt(1 - A^2) sin chi + A cos chi).
    The global sign is immaterial (data are formed with the same C).
    """
    lam = electron_wavelength_A(kv)
    cs = cs_mm * 1e7
    chi = np.pi * lam * defocus_A * s2 - 0.5 * np.pi * cs * lam ** 3 * s2 * s2
    return -(np.sqrt(1.0 - amp * amp) * np.sin(chi) + amp * np.cos(chi))


def ctf_pixels(q, defocus_A: float, M: int, ctf) -> np.ndarray:
    """CTF values C_i at pixels with kx^2+ky^2 = q; ones when ``ctf`` is None.

    ``ctf`` = dict(kv=..., cs_mm=..., amp=..., pixel_A=...).  Spatial
    frequency s = sqrt(q) / (M * pixel_A).
    """
    q = np.asarray(q, dtype=np.float64)
    if ctf is None:
        return np.ones_like(q)
    s2 = q / (M * ctf["pixel_A"]) ** 2
    return ctf_of_s2(s2, defocus_A, ctf["kv"], ctf["cs_mm"], ctf["amp"])
