"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula: each checks an oracle function
against an independent fact (a published value, a closed form, an invariant
relating two separately written functions, or brute force on tiny inputs).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2311_16100_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CTF = dict(kv=300.0, cs_mm=2.7, amp=0.1, pixel_A=1.5)


def rots(n, seed):
    return O.quat_to_rot(synth.shoemake_quaternions(n, seed)).astype(np.float32)


def cplx(shape, seed):
    return synth.complex_normal(shape, seed)


def read_golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ------------------------------------------------------------- generators
def test_splitmix64_published_vector():
    want = [int(r[0]) for r in read_golden("splitmix64_seed1234567.txt")]
    got = O.splitmix64(1234567, np.arange(5)).tolist()
    assert got == want


def test_rademacher_balanced_and_independent():
    Z = O.rademacher_probes(seed=7, block=3, n_vox=1 << 16, n_probes=32)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 0.01
    C = (Z @ Z.T) / Z.shape[1]
    off = C[~np.eye(32, dtype=bool)]
    assert np.max(np.abs(off)) < 0.03      # ~ 1/sqrt(65536) scale
    # different blocks give different probes
    Z2 = O.rademacher_probes(seed=7, block=4, n_vox=1 << 16, n_probes=32)
    assert abs(np.mean(Z * Z2)) < 0.01


# -------------------------------------------------------------- rotations
def hamilton(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_quat_to_rot_matches_sandwich_product():
    qs = synth.shoemake_quaternions(50, 11)
    g = np.random.default_rng(0)
    for q in qs:
        R = O.quat_to_rot(q)
        v = g.normal(size=3)
        qc = q * np.array([1, -1, -1, -1])
        rv = hamilton(hamilton(q, np.r_[0.0, v]), qc)[1:]
        np.testing.assert_allclose(R @ v, rv, atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1) < 1e-12


def test_quat_to_rot_axis_rotation():
    c = np.sqrt(0.5)
    R = O.quat_to_rot(np.array([c, 0, 0, c]))          # +90 deg about z
    np.testing.assert_allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(R @ [0, 1, 0], [-1, 0, 0], atol=1e-15)


# -------------------------------------------------------------------- CTF
def test_electron_wavelength_textbook():
    for kv, lam in read_golden("electron_wavelength.txt"):
        assert round(O.electron_wavelength_A(float(kv)), 4) == float(lam)


def test_ctf_zeros_and_limits():
    lam = O.electron_wavelength_A(300.0)
    df = 20000.0
    # Cs = 0, A = 0: C = -sin(pi lam df s^2), zero at s^2 = n / (lam df)
    for n in range(1, 6):
        s2 = n / (lam * df)
        assert abs(O.ctf_of_s2(s2, df, 300.0, 0.0, 0.0)) < 1e-9
        # and extremal (|C| = 1) halfway between zeros
        s2h = (n + 0.5) / (lam * df)
        assert abs(abs(O.ctf_of_s2(s2h, df, 300.0, 0.0, 0.0)) - 1) < 1e-9
    # pure amplitude contrast at DC
    assert abs(O.ctf_of_s2(0.0, df, 300.0, 2.7, 0.1) + 0.1) < 1e-15
    # |C| <= 1 everywhere
    s2 = np.linspace(0, 0.2, 1001)
    assert np.all(np.abs(O.ctf_of_s2(s2, df, 300.0, 2.7, 0.1)) <= 1 + 1e-12)


# ------------------------------------------------------------ projection
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_identity_rotation_is_central_plane(interp):
    M = 16
    v = cplx((M, M, M), 1)
    y = O.slice_project(v, np.eye(3, dtype=np.float32)[None], [0.0], M, M // 2 - 1,
                        interp, None)[0]
    m = O.disc_mask(M, M // 2 - 1).reshape(M, M)
    np.testing.assert_allclose(y[m], v[M // 2][m], atol=1e-14)
    assert np.all(y[~m] == 0)


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_quarter_turn_about_x_permutes_grid(interp):
    M = 16
    h = M // 2
    v = cplx((M, M, M), 2)
    R = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], dtype=np.float32)
    y = O.slice_project(v, R[None], [0.0], M, h - 1, interp, None)[0]
    # R^T (kx, ky, 0) = (kx, 0, -ky): pixel (iy, ix) reads voxel (z=-ky, y=0, x=kx)
    for iy in range(M):
        for ix in range(M):
            kx, ky = ix - h, iy - h
            if kx * kx + ky * ky <= (h - 1) ** 2:
                assert abs(y[iy, ix] - v[-ky + h, h, kx + h]) < 1e-14


def affine_volume(M, a, b):
    k = np.arange(M) - M // 2
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    return a[0] * kx + a[1] * ky + a[2] * kz + b


def test_trilinear_reproduces_affine_volumes():
    """Trilinear interpolation is exact for affine functions: pins the weights,
    the index <-> frequency map and the direction of the rotation (R^T r)."""
    M = 24
    h = M // 2
    a = np.array([0.3 + 1j, -2.0 + 0.5j, 1.25 - 0.7j])
    b = 0.1 - 0.2j
    v = affine_volume(M, a, b)
    R = rots(6, 3)
    y = O.slice_project(v, R, np.zeros(6), M, h - 1, "trilinear", None)
    kx, ky = O.pixel_coords(M)
    m = O.disc_mask(M, h - 1)
    for i in range(6):
        pts = (R[i].astype(np.float64).T @ np.stack([kx, ky, 0 * kx])).T   # R^T r
        want = pts @ a + b
        np.testing.assert_allclose(y[i].ravel()[m], want[m], atol=1e-11)


def test_nearest_matches_bruteforce_argmin():
    """k*(j) = argmin_k |r_k - R^T r_j| over all grid points (Definition 2.1),
    by exhaustive search; only near-ties may differ."""
    M = 8
    h = M // 2
    k = np.arange(M) - h
    kz, ky3, kx3 = np.meshgrid(k, k, k, indexing="ij")
    grid = np.stack([kx3.ravel(), ky3.ravel(), kz.ravel()], axis=1).astype(np.float64)
    for R in rots(10, 5):
        pix, vox, w = O.stencil(R, M, h - 1, "nearest")
        kx, ky = O.pixel_coords(M)
        pts = (R.astype(np.float64).T @ np.stack([kx[pix], ky[pix], 0 * pix])).T
        for p, t in enumerate(pts):
            d2 = np.sum((grid - t) ** 2, axis=1)
            best = np.argmin(d2)
            frac = np.abs(t - np.round(t))
            if np.all(np.abs(frac - 0.5) > 1e-5):
                assert vox[p, 0] == best


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("ctf", [None, CTF])
def test_adjoint_identity(interp, ctf):
    M = 12
    B = 5
    R = rots(B, 8)
    df = synth.defocus_angstrom(B, 9)
    x = cplx((M, M, M), 10)
    y = cplx((B, M, M), 11)
    Px = O.slice_project(x, R, df, M, M // 2 - 1, interp, ctf)
    Pty = O.backproject_adjoint(y, R, df, M, M // 2 - 1, interp, ctf)
    lhs = np.vdot(y, Px)          # <Px, y> with conjugate on y
    rhs = np.vdot(Pty, x)         # <x, P* y>
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------- objective
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_gradient_matches_central_differences(interp):
    """f is quadratic, so the central difference equals the directional
    derivative Re<g, e> up to rounding, for any step h."""
    M, B = 10, 4
    R = rots(B, 12)
    df = synth.defocus_angstrom(B, 13)
    x = cplx((B, M, M), 14)
    v = cplx((M, M, M), 15)
    lam, scale = 0.37, 2.5
    f, g = O.loss_grad(v, x, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
    f2 = O.loss(v, x, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
    assert abs(f - f2) <= 1e-12 * abs(f)
    for s in range(4):
        e = cplx((M, M, M), 100 + s)
        h = 1e-3
        fp = O.loss(v + h * e, x, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
        fm = O.loss(v - h * e, x, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
        fd = (fp - fm) / (2 * h)
        dd = np.sum((np.conj(g) * e).real)
        assert abs(fd - dd) <= 1e-8 * (abs(dd) + abs(f) * 1e-3)


def test_loss_zero_residual_at_generating_volume():
    M, B = 10, 3
    R = rots(B, 16)
    df = synth.defocus_angstrom(B, 17)
    v = cplx((M, M, M), 18)
    x = O.slice_project(v, R, df, M, M // 2 - 1, "trilinear", CTF)
    f, g = O.loss_grad(v, x, R, df, M, M // 2 - 1, "trilinear", CTF, 0.0, 1.0)
    assert abs(f) < 1e-20 and np.max(np.abs(g)) < 1e-12


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_hvp_is_the_gradients_linear_part(interp):
    """grad f(v) - grad f(0) = H v for both real and imaginary parts: ties the
    separately written HVP (C^2) to the gradient (C (C P v - x))."""
    M, B = 10, 4
    R = rots(B, 19)
    df = synth.defocus_angstrom(B, 20)
    x = cplx((B, M, M), 21)
    v = cplx((M, M, M), 22)
    lam, scale = 0.1, 3.0
    _, g1 = O.loss_grad(v, x, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
    _, g0 = O.loss_grad(0 * v, x, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
    Hr = O.hvp(v.real, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
    Hi = O.hvp(v.imag, R, df, M, M // 2 - 1, interp, CTF, lam, scale)
    np.testing.assert_allclose(g1 - g0, Hr + 1j * Hi, atol=1e-10 * np.max(np.abs(g1)))


def test_quadratic_model_along_a_direction():
    """f(v - eta d) = f(v) - eta Re<g, d> + eta^2/2 <d, H d>: the identity the
    closed-form Armijo step rests on, checked from loss, gradient and HVP."""
    M, B = 10, 4
    R = rots(B, 23)
    df = synth.defocus_angstrom(B, 24)
    x = cplx((B, M, M), 25)
    v = cplx((M, M, M), 26)
    d = cplx((M, M, M), 27)
    lam, scale = 0.2, 1.7
    f0, g = O.loss_grad(v, x, R, df, M, M // 2 - 1, "trilinear", CTF, lam, scale)
    Q = (np.sum(d.real * O.hvp(d.real, R, df, M, M // 2 - 1, "trilinear", CTF, lam, scale))
         + np.sum(d.imag * O.hvp(d.imag, R, df, M, M // 2 - 1, "trilinear", CTF, lam, scale)))
    for eta in (0.1, 0.7, 2.0):
        f1 = O.loss(v - eta * d, x, R, df, M, M // 2 - 1, "trilinear", CTF, lam, scale)
        model = f0 - eta * np.sum((np.conj(g) * d).real) + 0.5 * eta * eta * Q
        assert abs(f1 - model) <= 1e-11 * abs(f0)


def test_dense_hessian_symmetric_pd_and_diag():
    M, B = 4, 6
    R = rots(B, 28)
    df = synth.defocus_angstrom(B, 29)
    lam = 0.05
    H = O.dense_hessian(R, df, M, 1, "trilinear", CTF, lam, 1.0)
    np.testing.assert_allclose(H, H.T, atol=1e-13)
    assert np.min(np.linalg.eigvalsh(H)) >= lam - 1e-12
    d = O.exact_diag(R, df, M, 1, "trilinear", CTF, lam, 1.0).ravel()
    np.testing.assert_allclose(np.diag(H), d, atol=1e-13)


def test_exact_diag_nearest_counts_pixels():
    """Nearest, no CTF: diag(H)_j - lam = number of (image, pixel) pairs whose
    nearest grid point is j (Eq. pp / H diag), found by exhaustive argmin."""
    M, B = 8, 6
    h = M // 2
    R = rots(B, 30)
    lam = 1e-3
    d = O.exact_diag(R, np.zeros(B), M, h - 1, "nearest", None, lam, 1.0).ravel()
    k = np.arange(M) - h
    kz, ky3, kx3 = np.meshgrid(k, k, k, indexing="ij")
    grid = np.stack([kx3.ravel(), ky3.ravel(), kz.ravel()], axis=1).astype(np.float64)
    count = np.zeros(M ** 3)
    kx, ky = O.pixel_coords(M)
    m = O.disc_mask(M, h - 1)
    for i in range(B):
        pts = (R[i].astype(np.float64).T @ np.stack([kx[m], ky[m], 0 * kx[m]])).T
        for t in pts:
            count[np.argmin(np.sum((grid - t) ** 2, axis=1))] += 1
    np.testing.assert_allclose(d - lam, count, atol=1e-12)
    # centre voxel is hit by every image exactly once (Assumption 3.1, part 2)
    centre = (h * M + h) * M + h
    assert d[centre] == B + lam


def test_proposition_3_1_bound():
    M, N = 16, 40
    lam = 1e-8
    R = rots(N, 31)
    d = O.exact_diag(R, np.zeros(N), M, M // 2 - 1, "nearest", None, lam, 1.0).ravel()
    assert abs(d.max() - (N + lam)) < 1e-9
    kappa = d.max() / d.min()
    assert kappa >= (N + lam) / (N / M + lam)


# ------------------------------------------------------------- Hutchinson
def test_hutchinson_exact_under_nearest():
    """Remark 3.3: with a diagonal H one Rademacher probe gives diag(H)."""
    M, B = 12, 7
    R = rots(B, 32)
    df = synth.defocus_angstrom(B, 33)
    lam, scale = 0.01, 4.0
    want = O.exact_diag(R, df, M, M // 2 - 1, "nearest", CTF, lam, scale)
    for K in (1, 5):
        got = O.hutchinson_diag(R, df, M, M // 2 - 1, "nearest", CTF, lam, scale,
                                K, seed=99, block=1)
        np.testing.assert_allclose(got, want, rtol=1e-13)


def test_hutchinson_unbiased_under_trilinear():
    """E[z (.) Hz] = diag(H), Var = (1/K) sum_{l != j} H_jl^2 (Rademacher):
    averaged over many probe blocks the z-scores must stay small."""
    M, B = 4, 5
    R = rots(B, 34)
    df = synth.defocus_angstrom(B, 35)
    lam = 0.1
    H = O.dense_hessian(R, df, M, 1, "trilinear", CTF, lam, 1.0)
    var1 = np.sum(H ** 2, axis=1) - np.diag(H) ** 2
    n_blocks, K = 48, 32
    acc = np.zeros(M ** 3)
    for blk in range(n_blocks):
        acc += O.hutchinson_diag(R, df, M, 1, "trilinear", CTF, lam, 1.0,
                                 K, seed=5, block=blk).ravel()
    est = acc / n_blocks
    sd = np.sqrt(var1 / (K * n_blocks))
    used = sd > 0
    z = (est - np.diag(H))[used] / sd[used]
    assert np.max(np.abs(z)) < 5.0
    assert abs(np.mean(z)) < 4.0 / np.sqrt(used.sum())
    np.testing.assert_allclose(est[~used], np.diag(H)[~used], rtol=1e-12)


def nearest_counts(R, M):
    """(image, pixel) pairs per voxel whose nearest grid point it is, by
    exhaustive argmin over the grid (Definition 2.1 literally)."""
    h = M // 2
    k = np.arange(M) - h
    kz, ky3, kx3 = np.meshgrid(k, k, k, indexing="ij")
    grid = np.stack([kx3.ravel(), ky3.ravel(), kz.ravel()], axis=1).astype(np.float64)
    count = np.zeros(M ** 3)
    kx, ky = O.pixel_coords(M)
    m = O.disc_mask(M, h - 1)
    for i in range(R.shape[0]):
        pts = (R[i].astype(np.float64).T @ np.stack([kx[m], ky[m], 0 * kx[m]])).T
        for t in pts:
            count[np.argmin(np.sum((grid - t) ** 2, axis=1))] += 1
    return count


def test_precomputed_preconditioner_nearest_is_the_full_diagonal():
    """Section 4's precomputed arm under nearest, no CTF: each probe gives a
    batch's diagonal exactly (Remark 3.3) and equal batches scaled by N/B
    average to the full-data diagonal |Omega_j| + lam, whatever the epochs."""
    M, N, B = 8, 6, 2
    R = rots(N, 40)
    lam = 1e-3
    want = nearest_counts(R, M) + lam
    for epochs in (1, 3):
        got = O.precomputed_preconditioner(R, None, M, M // 2 - 1, "nearest", None, lam, B,
                                           epochs, 1, seed=3).ravel()
        np.testing.assert_allclose(got, want, rtol=1e-12)
    # a short last batch carries scale N/|I_last|: batches {0..3} and {4, 5}
    c1, c2 = nearest_counts(R[:4], M), nearest_counts(R[4:], M)
    got = O.precomputed_preconditioner(R, None, M, M // 2 - 1, "nearest", None, lam, 4, 2,
                                       3, seed=3).ravel()
    np.testing.assert_allclose(got, 0.5 * (lam + 1.5 * c1) + 0.5 * (lam + 3.0 * c2),
                               rtol=1e-12)


def test_precomputed_preconditioner_unbiased_under_trilinear():
    """Trilinear: the average of many batch estimates is unbiased for the
    full-data diagonal (z-scores against the dense Hessian, whose per-probe
    variance is sum_{l != j} H_jl^2 within each batch)."""
    M, N, B, E, K = 4, 6, 3, 16, 32
    R = rots(N, 41)
    df = synth.defocus_angstrom(N, 42)
    lam = 0.1
    H = O.dense_hessian(R, df, M, 1, "trilinear", CTF, lam, 1.0)
    # per-batch Hessians at scale N/B, to get the estimator's variance
    var = np.zeros(M ** 3)
    for sl in (slice(0, 3), slice(3, 6)):
        Hb = O.dense_hessian(R[sl], df[sl], M, 1, "trilinear", CTF, lam, N / B)
        var += (np.sum(Hb ** 2, axis=1) - np.diag(Hb) ** 2) / K
    n_it = E * (N // B)
    var = var / (N // B) / n_it
    est = O.precomputed_preconditioner(R, df, M, 1, "trilinear", CTF, lam, B, E, K,
                                       seed=8).ravel()
    sd = np.sqrt(var)
    used = sd > 0
    z = (est - np.diag(H))[used] / sd[used]
    assert np.max(np.abs(z)) < 5.0
    np.testing.assert_allclose(est[~used], np.diag(H)[~used], rtol=1e-12)


# ------------------------------------------------------------- in-plane shifts
def test_shift_phase_is_the_fourier_shift_theorem():
    """Integer shifts: multiplying the centred spectrum by T and transforming
    back rolls the real-space image by +t (numpy's FFT as the independent
    reference); T is unitary, T(0) = 1 and T(a) T(b) = T(a + b)."""
    M = 16
    g = np.random.default_rng(5)
    x = g.normal(size=(M, M))
    X = np.fft.fftshift(np.fft.fft2(x))          # index M/2 holds frequency 0
    for tx, ty in ((3, 0), (0, -5), (2, 7), (-8, 1)):
        T = O.shift_phase(M, [(tx, ty)])[0]
        y = np.fft.ifft2(np.fft.ifftshift(X * T)).real
        np.testing.assert_allclose(y, np.roll(x, (ty, tx), axis=(0, 1)), atol=1e-12)
    t1, t2 = (0.3, -1.7), (2.25, 0.5)
    T1, T2 = O.shift_phase(M, [t1])[0], O.shift_phase(M, [t2])[0]
    T12 = O.shift_phase(M, [(t1[0] + t2[0], t1[1] + t2[1])])[0]
    np.testing.assert_allclose(T1 * T2, T12, atol=1e-12)
    np.testing.assert_allclose(np.abs(T1), 1.0, rtol=1e-14)
    assert O.shift_phase(M, [(1.3, 2.1)])[0][M // 2, M // 2] == 1.0


def test_shifted_loss_equals_loss_on_corrected_images():
    """|x - C T S v| = |T* x - C S v| (T unitary, diagonal, commuting with C):
    the identity that lets the operators work with the unshifted slice."""
    M, B = 12, 4
    R = rots(B, 60)
    df = synth.defocus_angstrom(B, 61)
    v = cplx((M, M, M), 62)
    t = np.random.default_rng(63).uniform(-4, 4, size=(B, 2))
    x = cplx((B, M, M), 64)
    model = O.slice_project(v, R, df, M, M // 2 - 1, "trilinear", CTF)
    lhs = np.sum(np.abs(x - O.phase_shift(model, t, +1)) ** 2)
    rhs = np.sum(np.abs(O.phase_shift(x, t, -1) - model) ** 2)
    assert abs(lhs - rhs) <= 1e-12 * lhs


# ------------------------------------------------------- threshold alpha
def test_shell_ratio_asymptotics():
    """P_x(R)/P_v(R) ~ 2 pi R / (4 pi R^2) = 1/(2R) for 1-voxel shells (the
    lattice-point count of a thin annulus fluctuates by a few percent)."""
    for M, R in ((64, 31), (128, 63)):
        Px, Pv = O.shell_counts(M, R)
        assert abs(Px / Pv * 2 * R - 1) < 0.1
        assert abs(Px / (2 * np.pi * R) - 1) < 0.1
        assert abs(Pv / (4 * np.pi * R * R + np.pi / 3) - 1) < 0.05


def test_alpha_is_shell_mean_of_diag_for_uniform_poses():
    """Eq. (thresh value) is the expected Hessian entry in the shell of radius
    R for uniform orientations: compare with the mean of the exact diagonal
    over that shell, for shells lying inside the image disc."""
    M, N = 32, 400
    R = rots(N, 36)
    df = synth.defocus_angstrom(N, 37)
    lam = 1e-3
    r = M // 2 - 1
    k = np.arange(M) - M // 2
    q = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2).ravel()
    for ctf in (None, CTF):
        d = O.exact_diag(R, df, M, r, "nearest", ctf, lam, 1.0).ravel()
        ratios = []
        for Rs in range(3, 14):
            shell = (q >= Rs * Rs - Rs + 1) & (q <= Rs * Rs + Rs)
            a = O.alpha_threshold(df, M, r, ctf, lam, R=Rs)
            ratios.append(np.mean(d[shell]) / a)
        # single 1-voxel shells fluctuate with the lattice-point counts
        assert np.all(np.abs(np.array(ratios) - 1) < 0.25)
        assert abs(np.mean(ratios) - 1) < 0.06


# ------------------------------------------------------------ Algorithm 1
def test_alg1_step_is_em_m_step_under_nearest():
    """Remark 3.2: with nearest interpolation H is diagonal; with the exact
    diagonal as preconditioner, full batch and eta = 1, one step from any v
    lands on v* = H^{-1} b, the known-pose M-step."""
    M, B = 10, 12
    r = M // 2 - 1
    R = rots(B, 38)
    df = synth.defocus_angstrom(B, 39)
    x = cplx((B, M, M), 40)
    lam = 0.3
    D = O.exact_diag(R, df, M, r, "nearest", CTF, lam, 1.0)
    b = O.full_rhs(x, R, df, M, r, "nearest", CTF)
    v0 = cplx((M, M, M), 41)
    out = O.alg1_step(v0, D, np.zeros_like(D), 1.0, 1, x, R, df, M, r, "nearest",
                      CTF, lam, 1.0, alpha=1e-12, beta=0.9, c=0.4, mode="fixed")
    assert out["eta"] == 1.0 and out["halvings"] == 0
    np.testing.assert_allclose(out["v"], b / D, atol=1e-12 * np.max(np.abs(b / D)))


def test_alg1_armijo_accepts_largest_halving():
    """The accepted eta is the first eta_prev 2^-m with the Armijo condition,
    which for a quadratic is eta <= 2 (1 - c) G / Q."""
    M, B = 10, 6
    r = M // 2 - 1
    R = rots(B, 42)
    df = synth.defocus_angstrom(B, 43)
    x = cplx((B, M, M), 44)
    v = cplx((M, M, M), 45)
    lam, scale, c = 0.05, 3.0, 0.5
    for mode in ("plain", "hutchinson"):
        D = np.ones((M, M, M))
        out = O.alg1_step(v, D, np.zeros_like(D), 64.0, 1, x, R, df, M, r,
                          "trilinear", CTF, lam, scale, alpha=0.5, beta=0.9, c=c,
                          mode=mode, n_probes=8, seed=3)
        Dhat = np.maximum(np.abs(out["D"]), 0.5) if mode == "hutchinson" else np.ones_like(D)
        _, g = O.loss_grad(v, x, R, df, M, r, "trilinear", CTF, lam, scale)
        d = g / Dhat
        G = np.sum(np.abs(g) ** 2 / Dhat)
        Q = (np.sum(d.real * O.hvp(d.real, R, df, M, r, "trilinear", CTF, lam, scale))
             + np.sum(d.imag * O.hvp(d.imag, R, df, M, r, "trilinear", CTF, lam, scale)))
        bound = 2 * (1 - c) * G / Q
        assert out["eta"] <= bound < 2 * out["eta"]
        assert out["eta"] == 64.0 * 2.0 ** (-out["halvings"])


def test_cg_matches_nearest_closed_form():
    M, B = 10, 8
    r = M // 2 - 1
    R = rots(B, 46)
    df = synth.defocus_angstrom(B, 47)
    x = cplx((B, M, M), 48)
    lam = 0.2
    b = O.full_rhs(x, R, df, M, r, "nearest", CTF)
    vs, _ = O.cg_solve(b, R, df, M, r, "nearest", CTF, lam)
    D = O.exact_diag(R, df, M, r, "nearest", CTF, lam, 1.0)
    np.testing.assert_allclose(vs, b / D, atol=1e-10 * np.max(np.abs(b / D)))


# --------------------------------------- Algorithm 1's preconditioner update
def _alg1_run(batches, M, r, lam, scale, alpha, beta, steps, mode="hutchinson"):
    """Run alg1_step k = 1..steps on the given (x, R, df) batches in turn,
    collecting D_avg^(k), D^(k), the accepted eta and the step v - v+."""
    v = cplx((M, M, M), 50)
    D, Da, eta = np.ones((M, M, M)), np.zeros((M, M, M)), 1.0
    hist = []
    for k in range(1, steps + 1):
        x, R, df = batches[(k - 1) % len(batches)]
        out = O.alg1_step(v, D, Da, eta, k, x, R, df, M, r, "nearest", None, lam, scale,
                          alpha, beta, 0.5, mode, n_probes=3, seed=17)
        hist.append(dict(D_avg=out["D_avg"], D=out["D"], eta=out["eta"], v=v,
                         step=v - out["v"]))
        v, D, Da, eta = out["v"], out["D"], out["D_avg"], out["eta"]
    return hist


def test_alg1_preconditioner_update_closed_form_equal_batches():
    """Algorithm 1 (Eqs. hutch update and exp avg update) under nearest
    interpolation without CTF, the same batch at every iteration: H_I is
    diagonal, so every Rademacher estimate is exactly diag(H_I) (Remark 3.3),
    the running mean stays diag(H_I) and the exponential average from D^0 = I
    is D^(k) = beta^k + (1 - beta^k) diag(H_I).  A swapped beta / (1 - beta)
    or a running mean indexed from 0 fails this."""
    M, B = 10, 6
    r = M // 2 - 1
    R = rots(B, 51)
    x = cplx((B, M, M), 52)
    lam, scale, beta = 0.02, 3.0, 0.9
    diag = O.exact_diag(R, np.zeros(B), M, r, "nearest", None, lam, scale)
    hist = _alg1_run([(x, R, np.zeros(B))], M, r, lam, scale, 1e-9, beta, 5)
    for k, h in enumerate(hist, start=1):
        np.testing.assert_allclose(h["D_avg"], diag, rtol=1e-13)
        np.testing.assert_allclose(h["D"], beta ** k + (1 - beta ** k) * diag, rtol=1e-12)


def test_alg1_running_mean_over_different_batches():
    """Different batches I_1, I_2, I_3 (nearest, no CTF, so each estimate is
    the batch's exact diagonal): D_avg^(k) is the plain mean of the first k
    batch diagonals, and D^(k) = beta D^(k-1) + (1 - beta) D_avg^(k) from I."""
    M, B = 10, 5
    r = M // 2 - 1
    lam, scale, beta = 0.01, 4.0, 0.75
    batches = [(cplx((B, M, M), 60 + i), rots(B, 70 + i), np.zeros(B)) for i in range(3)]
    diags = [O.exact_diag(R, df, M, r, "nearest", None, lam, scale) for _, R, df in batches]
    hist = _alg1_run(batches, M, r, lam, scale, 1e-9, beta, 3)
    D = np.ones((M, M, M))
    for k, h in enumerate(hist, start=1):
        mean_k = sum(diags[:k]) / k
        np.testing.assert_allclose(h["D_avg"], mean_k, rtol=1e-13)
        D = beta * D + (1 - beta) * mean_k
        np.testing.assert_allclose(h["D"], D, rtol=1e-12)
    # the batch diagonals really differ, so the mean is not trivially one of them
    assert np.max(np.abs(diags[0] - diags[1])) > 1.0


def test_alg1_step_divides_by_thresholded_d():
    """Eq. thresh and the step of Algorithm 1: v+ = v - eta g / max(|D|, alpha),
    with g the mini-batch gradient (pinned by finite differences) and D the
    closed form above; alpha is set between the smallest and largest D so
    that both branches of the maximum occur."""
    M, B = 10, 6
    r = M // 2 - 1
    R = rots(B, 53)
    x = cplx((B, M, M), 54)
    lam, scale, beta = 0.02, 3.0, 0.9
    diag = O.exact_diag(R, np.zeros(B), M, r, "nearest", None, lam, scale)
    D1 = beta + (1 - beta) * diag
    alpha = float(0.5 * (D1.min() + D1.max()))
    hist = _alg1_run([(x, R, np.zeros(B))], M, r, lam, scale, alpha, beta, 1)
    h = hist[0]
    _, g = O.loss_grad(h["v"], x, R, np.zeros(B), M, r, "nearest", None, lam, scale)
    Dhat = np.where(D1 < alpha, alpha, D1)
    assert 0 < np.count_nonzero(D1 < alpha) < D1.size
    np.testing.assert_allclose(h["step"], h["eta"] * g / Dhat,
                               atol=1e-12 * np.max(np.abs(h["step"])))
    # plain mode: D-hat = I
    hp = _alg1_run([(x, R, np.zeros(B))], M, r, lam, scale, alpha, beta, 1, mode="plain")[0]
    np.testing.assert_allclose(hp["step"], hp["eta"] * g,
                               atol=1e-12 * np.max(np.abs(hp["step"])))


# ------------------------------------------------ per-voxel network features
def test_coverage_features_nearest_are_pixel_counts():
    """Nearest without CTF every weight is 1: the coverage count is the
    brute-force-pinned diagonal count |Omega_j| (exact_diag with lam = 0,
    scale 1) and the CTF^2 sum equals it (C = 1)."""
    M, B = 10, 7
    r = M // 2 - 1
    R = rots(B, 55)
    cov, c2 = O.coverage_features(R, np.zeros(B), M, r, "nearest", None)
    counts = O.exact_diag(R, np.zeros(B), M, r, "nearest", None, 0.0, 1.0)
    np.testing.assert_array_equal(cov, counts)
    np.testing.assert_array_equal(c2, counts)
    assert cov.sum() == B * int(np.count_nonzero(O.disc_mask(M, r)))


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_coverage_features_conserve_pixel_mass(interp):
    """The weights of a pixel sum to one (Definition 2.1's interpolation
    reproduces constants), so sum_j coverage_j = B n_px and
    sum_j ctf2w_j = sum_i sum_p C_ip^2 with C from the pinned CTF formula."""
    M, B = 12, 5
    r = M // 2 - 1
    R = rots(B, 56)
    df = synth.defocus_angstrom(B, 57)
    cov, c2 = O.coverage_features(R, df, M, r, interp, CTF)
    m = O.disc_mask(M, r)
    kx, ky = O.pixel_coords(M)
    q = (kx * kx + ky * ky)[m]
    c2_total = sum(float(np.sum(O.ctf_pixels(q, df[i], M, CTF) ** 2)) for i in range(B))
    assert abs(cov.sum() - B * int(np.count_nonzero(m))) < 1e-9 * B * m.sum()
    assert abs(c2.sum() - c2_total) < 1e-9 * c2_total
    assert np.all(cov >= 0) and np.all(c2 >= 0) and np.all(c2 <= cov + 1e-12)


def test_network_features_radius_column_closed_form():
    """The first feature of voxel j = (iz M + iy) M + ix is
    |k| / (M/2) with k = (ix, iy, iz) - M/2, written out voxel by voxel; the
    other two are log1p of the given per-voxel sums in the same order."""
    import math
    M = 12
    h = M // 2
    g = np.random.default_rng(5)
    cov = g.uniform(0, 50, size=(M, M, M))
    c2 = g.uniform(0, 9, size=(M, M, M))
    F = O.mlp.features(M, cov, c2)
    assert F.shape == (M ** 3, 3)
    for j in list(g.integers(0, M ** 3, size=40)) + [0, (h * M + h) * M + h,
                                                     (h * M + h) * M, (h * M + h) * M + h + 3]:
        iz, rem = divmod(int(j), M * M)
        iy, ix = divmod(rem, M)
        want = math.sqrt((ix - h) ** 2 + (iy - h) ** 2 + (iz - h) ** 2) / h
        assert abs(F[j, 0] - want) < 1e-15
        assert abs(F[j, 1] - math.log(1 + cov[iz, iy, ix])) < 1e-13
        assert abs(F[j, 2] - math.log(1 + c2[iz, iy, ix])) < 1e-13
    assert F[(h * M + h) * M + h, 0] == 0.0          # the centre, k = 0
    assert F[(h * M + h) * M, 0] == 1.0               # k = (-M/2, 0, 0)
    assert abs(F[0, 0] - math.sqrt(3)) < 1e-15        # the corner (-M/2, -M/2, -M/2)


def test_lbfgs_ground_truth():
    """Section 4's ground-truth solver: L-BFGS on Eq. optim cp reaches the
    minimiser, i.e. the nearest-interpolation closed form b / diag(H), the
    CG solution under trilinear interpolation with CTF, and H v = b."""
    M, B = 10, 8
    r = M // 2 - 1
    R = rots(B, 80)
    df = synth.defocus_angstrom(B, 81)
    x = cplx((B, M, M), 82)
    lam = 0.2
    b = O.full_rhs(x, R, df, M, r, "nearest", CTF)
    v, _ = O.lbfgs_solve(b, R, df, M, r, "nearest", CTF, lam)
    D = O.exact_diag(R, df, M, r, "nearest", CTF, lam, 1.0)
    np.testing.assert_allclose(v, b / D, atol=1e-10 * np.max(np.abs(b / D)))
    b = O.full_rhs(x, R, df, M, r, "trilinear", CTF)
    v, it = O.lbfgs_solve(b, R, df, M, r, "trilinear", CTF, lam, max_iter=400)
    vc, _ = O.cg_solve(b, R, df, M, r, "trilinear", CTF, lam)
    np.testing.assert_allclose(v, vc, atol=1e-9 * np.max(np.abs(vc)))
    Hv = (O.hvp(v.real, R, df, M, r, "trilinear", CTF, lam, 1.0)
          + 1j * O.hvp(v.imag, R, df, M, r, "trilinear", CTF, lam, 1.0))
    assert np.linalg.norm(Hv - b) <= 1e-10 * np.linalg.norm(b)
    assert it < 400


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_hutchinson_rows_equal_the_full_estimate(interp):
    """hutchinson_diag_at (rows of Eq. hutch computed one by one, for checks
    at sampled voxels of full-size runs) equals the literal full estimate
    hutchinson_diag, K Hessian-vector products, at every voxel."""
    M, B = 10, 6
    r = M // 2 - 1
    R = rots(B, 90)
    df = synth.defocus_angstrom(B, 91)
    lam, scale, K = 0.05, 3.0, 8
    full = O.hutchinson_diag(R, df, M, r, interp, CTF, lam, scale, K, 21, 4).ravel()
    g = np.random.default_rng(7)
    sel = np.concatenate([g.choice(M ** 3, size=40, replace=False),
                          [((M // 2) * M + M // 2) * M + M // 2]])
    rows = O.hutchinson_diag_at(sel, R, df, M, r, interp, CTF, lam, scale, K, 21, 4)
    np.testing.assert_allclose(rows, full[sel], rtol=1e-12, atol=1e-12)


def test_network_features_at_selected_voxels_equal_the_full_grid():
    """features(..., idx) takes voxels by linear index (z-major) and gives the
    rows of the whole-grid features."""
    M = 10
    g = np.random.default_rng(7)
    cov, c2w = g.uniform(0, 50, (M, M, M)), g.uniform(0, 5, (M, M, M))
    X = O.mlp.features(M, cov, c2w)
    idx = np.concatenate([g.choice(M ** 3, 40, replace=False), [0, M ** 3 - 1]])
    np.testing.assert_array_equal(O.mlp.features(M, cov, c2w, idx), X[idx])

