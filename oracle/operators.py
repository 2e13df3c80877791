"""Oracle: forward model, adjoint, loss, gradient, Hessian (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Shapes: volume complex [M][M][M] (z, y, x), images complex [B][M][M],
rotations [B][3][3] (the float32 values the GPU path receives), defocus [B]
in Angstrom.  ``interp`` is "nearest" or "trilinear"; ``ctf`` is None or a
dict(kv, cs_mm, amp, pixel_A).  Pixels outside the disc of radius r_max are
not part of the model: the forward operator writes 0 there and the adjoint,
loss and gradient ignore them.
"""
from __future__ import annotations

import numpy as np

from .geometry import ctf_pixels, pixel_coords, stencil


def _image_terms(R, defocus, M, r_max, interp, ctf):
    """Stencil of P_i plus the CTF diagonal C_i on the used pixels."""
    pix, vox, w = stencil(R, M, r_max, interp)
    kx, ky = pixel_coords(M)
    C = ctf_pixels((kx * kx + ky * ky)[pix], defocus, M, ctf)
    return pix, vox, w, C


def slice_project(vol, R, defocus, M, r_max, interp, ctf):
    """y_i = C_i P_i v for every image (Eq. fwd model without noise).

    Definition 2.1: P^nn takes the nearest voxel, P^tri the trilinear
    combination of the eight surrounding voxels, of v at R_i^T r.
    """
    v = np.asarray(vol, dtype=np.complex128).ravel()
    B = len(R)
    out = np.zeros((B, M * M), dtype=np.complex128)
    for i in range(B):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        out[i, pix] = C * np.sum(w * v[vox], axis=1)
    return out.reshape(B, M, M)


def backproject_adjoint(images, R, defocus, M, r_max, interp, ctf, scale=1.0):
    """scale * sum_i P_i^* C_i y_i: the adjoint of ``slice_project``.

    P^* is the conjugate transpose of the (real-weight) interpolation matrix
    of Definition 2.1, so each used pixel adds w * C * y to each of its
    voxels.
    """
    y = np.asarray(images, dtype=np.complex128).reshape(len(R), M * M)
    g = np.zeros(M ** 3, dtype=np.complex128)
    for i in range(len(R)):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        contrib = (w * (C * y[i, pix])[:, None])
        np.add.at(g, vox.ravel(), contrib.ravel())
    return (scale * g).reshape(M, M, M)


def loss(vol, images, R, defocus, M, r_max, interp, ctf, lam, scale):
    """f_I(v) = scale/2 sum_i |x_i - C_i P_i v|^2 + lam/2 |v|^2.

    Eq. (optim cp) is the full-data objective (scale = 1).  For a mini-batch
    I of a dataset of N images we take scale = N/|I|, an unbiased estimate of
    the data term of that objective (Sections 2.3 and 3 scale the sum
    differently; this is our reading).
    """
    y = slice_project(vol, R, defocus, M, r_max, interp, ctf)
    x = np.asarray(images, dtype=np.complex128)
    r = np.zeros_like(y)
    for i in range(len(R)):
        pix, _, _, _ = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        r[i].ravel()[pix] = (y[i].ravel() - x[i].ravel())[pix]
    v = np.asarray(vol, dtype=np.complex128)
    return 0.5 * scale * np.sum(np.abs(r) ** 2) + 0.5 * lam * np.sum(np.abs(v) ** 2)


def loss_grad(vol, images, R, defocus, M, r_max, interp, ctf, lam, scale):
    """(f_I(v), grad f_I(v)) with grad = scale sum_i P_i^* C_i (C_i P_i v - x_i) + lam v.

    Identifying C^{M_v} with R^{2 M_v}, the gradient of Eq. (optim cp) in
    complex form is H v - b with H of Eq. (hessian) and b = sum_i P_i^* C_i x_i.
    """
    v = np.asarray(vol, dtype=np.complex128)
    x = np.asarray(images, dtype=np.complex128).reshape(len(R), M * M)
    g = np.zeros(M ** 3, dtype=np.complex128)
    data = 0.0
    vf = v.ravel()
    for i in range(len(R)):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        res = C * np.sum(w * vf[vox], axis=1) - x[i, pix]
        data += np.sum(np.abs(res) ** 2)
        np.add.at(g, vox.ravel(), (w * (C * res)[:, None]).ravel())
    f = 0.5 * scale * data + 0.5 * lam * np.sum(np.abs(v) ** 2)
    return f, (scale * g).reshape(M, M, M) + lam * v


def hvp(z, R, defocus, M, r_max, interp, ctf, lam, scale):
    """H_I z = scale sum_i P_i^* C_i^2 P_i z + lam z (Eq. hessian with CTF).

    ``z`` is real; the result is real since P has real weights and C is real.
    """
    zf = np.asarray(z, dtype=np.float64).ravel()
    out = np.zeros(M ** 3)
    for i in range(len(R)):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        y = C * C * np.sum(w * zf[vox], axis=1)
        np.add.at(out, vox.ravel(), (w * y[:, None]).ravel())
    return (scale * out + lam * zf).reshape(M, M, M)


def exact_diag(R, defocus, M, r_max, interp, ctf, lam, scale):
    """diag(H_I)_j = lam + scale sum_i sum_p C_ip^2 w_pj^2.

    The diagonal of Eq. (hessian): the (j, j) entry of P^* C^2 P sums the
    squared weight of voxel j in every row of P, times C^2.  Under nearest
    interpolation without CTF this is |Omega_j| + lam (Eq. H diag) when each
    image maps to voxel j at most once.
    """
    out = np.zeros(M ** 3)
    for i in range(len(R)):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        np.add.at(out, vox.ravel(), (w * w * (C * C)[:, None]).ravel())
    return (scale * out + lam).reshape(M, M, M)


def coverage_features(R, defocus, M, r_max, interp, ctf):
    """Per-voxel sums (sum_i sum_p w_pj, sum_i sum_p C_ip^2 w_pj).

    The first is the pose-coverage count |Omega_j| of Section 3.1 under
    nearest interpolation (one hit per image), a soft count otherwise; the
    second is the accumulated CTF^2 seen by the voxel.
    """
    cov = np.zeros(M ** 3)
    c2 = np.zeros(M ** 3)
    for i in range(len(R)):
        pix, vox, w, C = _image_terms(R[i], defocus[i], M, r_max, interp, ctf)
        np.add.at(cov, vox.ravel(), w.ravel())
        np.add.at(c2, vox.ravel(), (w * (C * C)[:, None]).ravel())
    return cov.reshape(M, M, M), c2.reshape(M, M, M)


def dense_hessian(R, defocus, M, r_max, interp, ctf, lam, scale):
    """H_I as a dense [M^3][M^3] matrix, column j = H_I e_j (tiny M only)."""
    n = M ** 3
    H = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        H[:, j] = hvp(e, R, defocus, M, r_max, interp, ctf, lam, scale).ravel()
    return H
