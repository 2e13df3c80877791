"""Pins of the oracle's diagnostics (Fourier shell correlation, per-shell
statistics, conditioning by radius) against facts that do not come from the
oracle itself: number theory, algebraic identities of Eq. fsc, the
inequalities of Proposition 3.1 / Eq. cond number p, brute force."""
import numpy as np

import oracle as O
from oracle import diagnostics as Dg
from paper_2311_16100_gb300 import synth


def cplx(shape, seed):
    g = np.random.default_rng(seed)
    return g.normal(size=shape) + 1j * g.normal(size=shape)


def sum_of_three_squares(q):
    """Legendre's three-square theorem: q is a sum of three squares unless
    q = 4^a (8b + 7)."""
    while q > 0 and q % 4 == 0:
        q //= 4
    return q % 8 != 7


def test_shells_agree_with_the_integer_shell_rule():
    """round(|k|) shells counted two independent ways (floating rounding vs the
    integer inequalities R^2 - R + 1 <= |k|^2 <= R^2 + R)."""
    for M in (16, 32):
        s = Dg.shell_index(M)
        for R in range(1, M // 2):
            assert int(np.sum(s == R)) == O.shell_counts(M, R)[1]
        assert int(np.sum(s == 0)) == 1


def test_shell_min_max_of_the_squared_radius_follow_number_theory():
    """For x = |k|^2 the smallest / largest value in shell r is the smallest /
    largest integer of [r^2 - r + 1, r^2 + r] that is a sum of three squares."""
    M = 32
    k = np.arange(M) - M // 2
    q = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2).astype(float)
    n = M // 2 - 1           # shells whose every lattice point lies on the grid
    lo, hi, cnt = Dg.shell_minmax(q, M, n)
    for r in range(1, n):
        cands = [t for t in range(r * r - r + 1, r * r + r + 1) if sum_of_three_squares(t)]
        assert lo[r] == min(cands) and hi[r] == max(cands)
    assert lo[0] == hi[0] == 0 and cnt[0] == 1
    k8 = np.arange(8) - 4
    q8 = k8[:, None, None] ** 2 + k8[None, :, None] ** 2 + k8[None, None, :] ** 2
    lo, hi, cnt = Dg.shell_minmax(q8, 8, 20)         # shells beyond the grid are empty
    assert np.all(cnt[8:] == 0) and np.all(np.isinf(lo[8:])) and np.all(hi[8:] == -np.inf)


def test_fsc_identities():
    """Eq. fsc: 1 for identical volumes and for positive multiples, -1 for a
    sign flip, cos(theta) for a global phase, and each shell depends on that
    shell only; the |u|^2 sums partition the energy."""
    M = 16
    u = cplx((M, M, M), 1)
    n = 14
    one, sums = Dg.fsc(u, u, M, n)
    np.testing.assert_allclose(one, 1.0, rtol=1e-14)
    np.testing.assert_allclose(Dg.fsc(u, 3.0 * u, M, n)[0], 1.0, rtol=1e-14)
    np.testing.assert_allclose(Dg.fsc(u, -u, M, n)[0], -1.0, rtol=1e-14)
    th = 0.7
    np.testing.assert_allclose(Dg.fsc(u, np.exp(1j * th) * u, M, n)[0], np.cos(th), rtol=1e-13)
    v = cplx((M, M, M), 2)
    f0 = Dg.fsc(u, v, M, n)[0]
    s = Dg.shell_index(M)
    w = v.copy()
    w[s == 5] *= 2.5                 # scaling one shell changes no FSC value
    np.testing.assert_allclose(Dg.fsc(u, w, M, n)[0], f0, rtol=1e-12)
    w[s == 5] = u[s == 5]            # replacing it sets that shell to 1 only
    f1 = Dg.fsc(u, w, M, n)[0]
    assert abs(f1[5] - 1) < 1e-14
    np.testing.assert_allclose(np.delete(f1, 5), np.delete(f0, 5), rtol=1e-12)
    big = int(s.max()) + 1
    _, sums = Dg.fsc(u, v, M, big)
    np.testing.assert_allclose(sums[:, 1].sum(), np.sum(np.abs(u) ** 2), rtol=1e-12)


def test_fsc_of_independent_noise_is_near_zero():
    """Independent complex Gaussian volumes: FSC(r) has mean 0 and standard
    deviation about 1/sqrt(2 |S_r|)."""
    M = 32
    u, v = cplx((M, M, M), 3), cplx((M, M, M), 4)
    f, _ = Dg.fsc(u, v, M, M // 2)
    n = np.bincount(Dg.shell_index(M).ravel())[: M // 2]
    z = f[1:] * np.sqrt(2 * n[1:])
    assert np.max(np.abs(z)) < 4.5


def test_p_ratio_asymptotics():
    """p(R) -> (pi R^2) / (4/3 pi R^3) = 3 / (4R) (the paper's approximation)."""
    for R in (20, 40, 60):
        assert abs(Dg.p_ratio(128, R) * 4 * R / 3 - 1) < 0.05


def test_condition_by_radius_under_nearest():
    """Nearest, no CTF, uniform poses: kappa(R) equals the brute-force max/min
    of diag(H) over round(|k|) <= R, never decreases with R, and obeys the
    lower bound of Eq. cond number p; with few images some voxel of a large
    ball is never hit, so the minimum is lam (Proposition 3.1, M > N case)."""
    M, lam = 24, 1e-3
    for N in (3, 60):
        R = O.quat_to_rot(synth.shoemake_quaternions(N, 50 + N))
        d = O.exact_diag(R, np.zeros(N), M, M // 2 - 1, "nearest", None, lam, 1.0)
        radii = list(range(1, M // 2))
        kap = Dg.condition_by_radius(d, M, radii)
        k = np.arange(M) - M // 2
        rr = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
        for Rk, kv in zip(radii, kap):
            ball = rr < Rk + 0.5
            assert kv == d[ball].max() / d[ball].min()
        assert np.all(np.diff(kap) >= 0)
        for Rk, kv in zip(radii, kap):
            p = Dg.p_ratio(M, Rk)
            if 1 / p <= N:
                assert kv >= Dg.kappa_lower_bound(N, lam, p) * (1 - 1e-12)
        if N == 3:
            assert d.min() == lam and kap[-1] >= (N + lam) / lam
