"""Parity of the per-shell kernels (Fourier shell correlation, shell
minimum / maximum) and of the in-plane shift phase with the oracle."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as Dg
from cryo_cases import Case, rel_l2
from paper_2311_16100_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300.ops import Handle
    hd = Handle(0)
    yield hd
    hd.close()


def cplx(M, seed):
    g = np.random.default_rng(seed)
    return (g.normal(size=(M, M, M)) + 1j * g.normal(size=(M, M, M))).astype(np.complex64)


@pytest.mark.parametrize("M,n", [(4, 4), (16, 14), (30, 16), (64, 40), (128, 64)])
def test_fsc_matches_oracle(h, M, n):
    u = cplx(M, M)
    v = (0.5 * u + cplx(M, M + 1)).astype(np.complex64)
    d = torch.device("cuda")
    f, sums = h.fsc(torch.from_numpy(u).to(d), torch.from_numpy(v).to(d), n)
    fo, so = Dg.fsc(u, v, M, n)
    np.testing.assert_allclose(sums.cpu().numpy(), so, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(f.cpu().numpy(), fo, rtol=1e-9, atol=1e-12)


def test_fsc_of_a_volume_with_itself_and_empty_shells(h):
    M = 16
    u = torch.from_numpy(cplx(M, 9)).cuda()
    f, sums = h.fsc(u, u, 30)
    f = f.cpu().numpy()
    last = int(np.rint(np.sqrt(3 * (M // 2) ** 2)))   # corner (-M/2, -M/2, -M/2): shell 14
    np.testing.assert_allclose(f[: last + 1], 1.0, rtol=1e-12)
    assert np.all(f[last + 1:] == 0) and np.all(sums.cpu().numpy()[last + 1:] == 0)


@pytest.mark.parametrize("M,n", [(8, 20), (32, 16), (96, 84)])
def test_shell_minmax_matches_oracle_exactly(h, M, n):
    g = np.random.default_rng(M)
    x = g.normal(size=(M, M, M)).astype(np.float32)
    lo, hi, cnt = h.shell_minmax(torch.from_numpy(x).cuda(), n)
    lo_o, hi_o, cnt_o = Dg.shell_minmax(x, M, n)
    assert np.array_equal(lo.cpu().numpy().astype(np.float64), lo_o)
    assert np.array_equal(hi.cpu().numpy().astype(np.float64), hi_o)
    assert np.array_equal(cnt.cpu().numpy(), cnt_o)


def test_condition_by_radius_from_gpu_diagonal(h):
    """kappa(R) from cs_exact_diag + cs_shell_minmax vs the oracle's."""
    M, N, lam = 32, 200, 1e-3
    q = synth.shoemake_quaternions(N, 61)
    R = O.quat_to_rot(q).astype(np.float32)
    from paper_2311_16100_gb300.ops import Geometry
    geom = Geometry(M, M // 2 - 1, "nearest", None)
    d, _, _ = h.exact_diag(geom, torch.from_numpy(R).cuda(), None, lam, 1.0)
    lo, hi, _ = h.shell_minmax(d, M // 2)
    lo, hi = lo.cpu().numpy().astype(np.float64), hi.cpu().numpy().astype(np.float64)
    radii = list(range(1, M // 2))
    kap = [np.max(hi[: r + 1]) / np.min(lo[: r + 1]) for r in radii]
    want = Dg.condition_by_radius(O.exact_diag(R, np.zeros(N), M, M // 2 - 1, "nearest", None,
                                               lam, 1.0), M, radii)
    np.testing.assert_allclose(kap, want, rtol=1e-5)


def test_shell_kernels_reject_bad_arguments(h):
    from paper_2311_16100_gb300.ops import CryoSGDError
    u = torch.zeros((16, 16, 16), dtype=torch.complex64, device="cuda")
    for n in (0, 1025):
        with pytest.raises(CryoSGDError):
            h.fsc(u, u, n)
        with pytest.raises(CryoSGDError):
            h.shell_minmax(u.real.contiguous(), n)
    with pytest.raises(CryoSGDError):
        h.fsc(torch.zeros((15, 15, 15), dtype=torch.complex64, device="cuda"),
              torch.zeros((15, 15, 15), dtype=torch.complex64, device="cuda"), 4)


@pytest.mark.parametrize("M,B", [(16, 3), (30, 5), (128, 4)])
def test_phase_shift_matches_oracle(h, M, B):
    g = np.random.default_rng(M + B)
    x = (g.normal(size=(B, M, M)) + 1j * g.normal(size=(B, M, M))).astype(np.complex64)
    t = g.uniform(-M / 2, M / 2, size=(B, 2)).astype(np.float32)
    t[0] = (3.0, -7.0)                                # an integer shift
    d = torch.device("cuda")
    ts = torch.from_numpy(t).to(d)
    for sign in (1, -1):
        img = torch.from_numpy(x).to(d)
        h.phase_shift(img, ts, sign)
        want = O.phase_shift(x, t.astype(np.float64), sign)
        assert rel_l2(img.cpu().numpy(), want) <= 1e-6
    img = torch.from_numpy(x).to(d)
    h.phase_shift(img, ts, 1)
    h.phase_shift(img, ts, -1)
    assert rel_l2(img.cpu().numpy(), x) <= 1e-6


def test_gradient_with_shifts_through_corrected_images(h):
    """Images formed with shifts (forward model C T S v + noise) and corrected
    once with T*: the library's gradient equals the oracle's gradient of the
    shifted objective, computed as S* C (C S v - T* x)."""
    c = Case(32, 12, interp="trilinear", ctf=True, seed=71)
    t = np.random.default_rng(72).uniform(-6, 6, size=(12, 2)).astype(np.float32)
    x_shifted = O.phase_shift(c.images, t.astype(np.float64), +1).astype(np.complex64)
    g = c.to_gpu()
    img = torch.from_numpy(x_shifted).cuda()
    h.phase_shift(img, torch.from_numpy(t).cuda(), -1)
    v = torch.from_numpy((0.5 * c.vol).astype(np.complex64)).cuda()
    loss, grad = h.loss_grad(c.gpu_geometry(), v, img, g["rot"], g["df"], 0.01, 2.0)
    corrected = O.phase_shift(x_shifted, t.astype(np.float64), -1)
    want_l, want_g = O.loss_grad(0.5 * c.vol, corrected, c.R, c.df, lam=0.01, scale=2.0,
                                 **c.geo())
    assert rel_l2(grad.cpu().numpy(), want_g) <= 1e-4
    assert abs(float(loss) - want_l) <= 1e-4 * abs(want_l)


def test_phase_shift_rejects_bad_arguments(h):
    from paper_2311_16100_gb300.ops import CryoSGDError
    img = torch.zeros((2, 16, 16), dtype=torch.complex64, device="cuda")
    t = torch.zeros((2, 2), device="cuda")
    with pytest.raises(CryoSGDError):
        h.phase_shift(img, t, 0)
    with pytest.raises(CryoSGDError):
        h.phase_shift(torch.zeros((2, 15, 15), dtype=torch.complex64, device="cuda"), t, 1)
