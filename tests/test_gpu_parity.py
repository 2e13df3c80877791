"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: nearest-neighbour voxel indices bit-exact; slices relative L2
<= 1e-5; adjoint, gradient, Hessian-vector products and diag(H) relative L2
<= 1e-4 (FP32 arithmetic and FP32 atomic accumulation against FP64).
"""
import numpy as np
import pytest

import oracle as O
from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SLICE = 1e-5
TOL_GRAD = 1e-4


@pytest.fixture(scope="module", params=["vector", "vector_slabs3", "tiled", "pixel"])
def h(request):
    """A handle per scatter algorithm (and the vector traversal split into
    three z-slabs, as large grids run it): every parity test runs on each."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300.ops import Handle
    hd = Handle(0)
    if request.param == "vector_slabs3":
        hd.set_algo("vector")
        hd.set_slabs(3)
    else:
        hd.set_algo(request.param)
    hd.algo_name = request.param
    yield hd
    # reports a bounded wait that ran out and, in the debug variant of the
    # library, any device-side index range check that failed
    hd.check_device_status()
    hd.close()


def cpu(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ poses
def test_quat_to_rot(h):
    c = Case(8, 257, seed=1)
    g = c.to_gpu()
    R = cpu(h.quat_to_rot(g["quat"]))
    want = O.quat_to_rot(c.quat.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(R - want)) < 2e-6


# ------------------------------------------------------------ forward slice
@pytest.mark.parametrize("M,B", [(32, 37), (30, 11), (64, 9), (128, 3)])
def test_nearest_indices_bit_exact(h, M, B):
    """Volume whose value is its own linear index: the slice returns the
    chosen voxel of every pixel, compared exactly with the oracle's rule."""
    c = Case(M, B, interp="nearest", ctf=False, seed=M + B)
    idx = np.arange(M ** 3, dtype=np.float32).astype(np.complex64).reshape(M, M, M)
    g = c.to_gpu()
    vol = torch.from_numpy(idx).cuda()
    y = cpu(h.slice_project(c.gpu_geometry(), vol, g["rot"]))
    for i in range(B):
        pix, vox, w = O.stencil(c.R[i], M, c.r_max, "nearest")
        got = y[i].ravel()[pix].real.astype(np.int64)
        assert np.array_equal(got, np.where(w[:, 0] > 0, vox[:, 0], 0))
        rest = np.setdiff1d(np.arange(M * M), pix)
        assert np.all(y[i].ravel()[rest] == 0)


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("ctf", [False, True])
@pytest.mark.parametrize("M,B", [(32, 20), (30, 7), (64, 6)])
def test_slice_project(h, interp, ctf, M, B):
    c = Case(M, B, interp=interp, ctf=ctf, seed=3 * M + B)
    g = c.to_gpu()
    y = cpu(h.slice_project(c.gpu_geometry(), g["vol"], g["rot"], g["df"]))
    want = O.slice_project(c.vol, c.R, c.df, **c.geo())
    assert rel_l2(y, want) <= TOL_SLICE


def test_slice_project_small_disc_and_tiny_grid(h):
    for M, r in ((4, 1), (16, 3), (34, 16)):
        c = Case(M, 5, interp="trilinear", ctf=True, seed=M, r_max=r)
        g = c.to_gpu()
        y = cpu(h.slice_project(c.gpu_geometry(), g["vol"], g["rot"], g["df"]))
        want = O.slice_project(c.vol, c.R, c.df, **c.geo())
        assert rel_l2(y, want) <= TOL_SLICE


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("M,B", [(32, 40), (30, 9)])
def test_backproject_adjoint(h, interp, M, B):
    c = Case(M, B, interp=interp, ctf=True, seed=5 * M + B)
    g = c.to_gpu()
    out = cpu(h.backproject_adjoint(c.gpu_geometry(), g["images"], g["rot"], g["df"], scale=2.5))
    want = O.backproject_adjoint(c.images, c.R, c.df, scale=2.5, **c.geo())
    assert rel_l2(out, want) <= TOL_SLICE * 10


def test_backproject_accumulates_split_batches(h):
    c = Case(32, 30, seed=77)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    full = h.backproject_adjoint(geom, g["images"], g["rot"], g["df"])
    acc = torch.zeros_like(full)
    for a, b in ((0, 13), (13, 30)):
        h.backproject_adjoint(geom, g["images"][a:b].contiguous(), g["rot"][a:b].contiguous(),
                              g["df"][a:b].contiguous(), vol_accum=acc)
    assert rel_l2(cpu(acc), cpu(full)) <= 1e-6


# ------------------------------------------------------------ loss, gradient
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("ctf", [False, True])
@pytest.mark.parametrize("M,B", [(32, 50), (30, 13), (64, 8)])
def test_loss_grad(h, interp, ctf, M, B):
    c = Case(M, B, interp=interp, ctf=ctf, seed=7 * M + B)
    g = c.to_gpu()
    lam, scale = 0.05, 20.0
    v = (c.vol * 0.7 + 0.1).astype(np.complex64)
    vg = torch.from_numpy(v).cuda()
    loss, grad = h.loss_grad(c.gpu_geometry(), vg, g["images"], g["rot"], g["df"], lam, scale)
    f, gw = O.loss_grad(v, c.images, c.R, c.df, lam=lam, scale=scale, **c.geo())
    assert rel_l2(cpu(grad), gw) <= TOL_GRAD
    assert abs(float(loss) - f) <= 1e-6 * abs(f)


def test_loss_grad_empty_batch(h):
    c = Case(16, 0, seed=9)
    v = torch.from_numpy(c.vol).cuda()
    rot = torch.empty((0, 3, 3), device="cuda")
    img = torch.empty((0, 16, 16), dtype=torch.complex64, device="cuda")
    df = torch.empty((0,), device="cuda")
    loss, grad = h.loss_grad(c.gpu_geometry(), v, img, rot, df, 0.3, 1.0)
    np.testing.assert_allclose(cpu(grad), 0.3 * c.vol, rtol=1e-6)
    assert abs(float(loss) - 0.15 * np.sum(np.abs(c.vol.astype(np.complex128)) ** 2)) < 1e-6 * float(loss)


def test_loss_grad_deterministic_loss(h):
    c = Case(32, 64, seed=10)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    a = float(h.loss_grad(geom, g["vol"], g["images"], g["rot"], g["df"], 0.1, 3.0)[0])
    b = float(h.loss_grad(geom, g["vol"], g["images"], g["rot"], g["df"], 0.1, 3.0)[0])
    assert a == b


# ------------------------------------------------------------ Hessian terms
@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("M,B", [(32, 30), (30, 9)])
def test_hvp(h, interp, M, B):
    c = Case(M, B, interp=interp, ctf=True, seed=11 * M + B)
    g = c.to_gpu()
    z = np.random.default_rng(M).normal(size=(M, M, M)).astype(np.float32)
    Hz = cpu(h.hvp(c.gpu_geometry(), torch.from_numpy(z).cuda(), g["rot"], g["df"], 0.2, 4.0))
    want = O.hvp(z, c.R, c.df, lam=0.2, scale=4.0, **c.geo())
    assert rel_l2(Hz, want) <= TOL_GRAD


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
@pytest.mark.parametrize("K", [1, 7, 16, 32])
def test_hutchinson_diag(h, interp, K):
    M, B = (32, 24) if interp == "trilinear" else (30, 17)
    c = Case(M, B, interp=interp, ctf=True, seed=13 * K + M)
    g = c.to_gpu()
    lam, scale = 0.01, 8.0
    d = cpu(h.hutchinson_diag(c.gpu_geometry(), g["rot"], g["df"], lam, scale, n_probes=K,
                              seed=1234, probe_block=3))
    want = O.hutchinson_diag(c.R, c.df, lam=lam, scale=scale, n_probes=K, seed=1234, block=3,
                             **c.geo())
    assert rel_l2(d, want) <= TOL_GRAD


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_exact_diag_and_features(h, interp):
    c = Case(32, 40, interp=interp, ctf=True, seed=17)
    g = c.to_gpu()
    d, cov, cw = h.exact_diag(c.gpu_geometry(), g["rot"], g["df"], 0.02, 3.0, True, True, True)
    want = O.exact_diag(c.R, c.df, lam=0.02, scale=3.0, **c.geo())
    cov_w, c2_w = O.coverage_features(c.R, c.df, **c.geo())
    cov_w, c2_w = 3.0 * cov_w, 3.0 * c2_w          # the batch's sums at scale 3
    assert rel_l2(cpu(d), want) <= TOL_GRAD
    assert rel_l2(cpu(cw), c2_w) <= TOL_GRAD
    if interp == "nearest":
        assert np.array_equal(cpu(cov), cov_w)        # integer counts, exact
    else:
        assert rel_l2(cpu(cov), cov_w) <= TOL_GRAD


def test_hutchinson_equals_exact_diag_under_nearest(h):
    c = Case(40, 25, interp="nearest", ctf=True, seed=19)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    hd = cpu(h.hutchinson_diag(geom, g["rot"], g["df"], 0.1, 2.0, n_probes=1, seed=5))
    ed = cpu(h.exact_diag(geom, g["rot"], g["df"], 0.1, 2.0)[0])
    assert rel_l2(hd, ed) <= 1e-6


@pytest.mark.parametrize("interp", ["nearest", "trilinear"])
def test_precompute_preconditioner(h, interp):
    """Section 4's precomputed arm: running mean of batch estimates over
    epochs, a short last batch with its own scale, probe block = iteration."""
    c = Case(24, 20, interp=interp, ctf=True, seed=29)
    g = c.to_gpu()
    lam = 0.05
    D = torch.full((24, 24, 24), float("nan"), device="cuda")   # never read
    h.precompute_preconditioner(c.gpu_geometry(), g["rot"], g["df"], B=8, n_epochs=2, lam=lam,
                                n_probes=4, seed=77, out=D)
    want = O.precomputed_preconditioner(c.R, c.df, c.M, c.r_max, c.interp, c.ctf, lam, 8, 2, 4,
                                        seed=77)
    assert rel_l2(cpu(D), want) <= TOL_GRAD


def test_precompute_preconditioner_rejects_bad_arguments(h):
    from paper_2311_16100_gb300.ops import CryoSGDError
    c = Case(16, 4, seed=31)
    g = c.to_gpu()
    for kw in (dict(B=0), dict(n_epochs=0), dict(n_probes=33)):
        args = dict(B=2, n_epochs=1, n_probes=4)
        args.update(kw)
        with pytest.raises(CryoSGDError):
            h.precompute_preconditioner(c.gpu_geometry(), g["rot"], g["df"], **args)


def test_threshold_alpha(h):
    for ctf in (False, True):
        c = Case(64, 300, ctf=ctf, seed=23)
        g = c.to_gpu()
        a = float(h.threshold_alpha(c.gpu_geometry(), g["df"], 300, 1e-3, 2.0))
        want = O.alpha_threshold(c.df, c.M, c.r_max, c.ctf, 1e-3, scale_alpha=2.0)
        assert abs(a - want) <= 1e-5 * want


# ------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("mode,interp,M", [("hutchinson", "trilinear", 24),
                                           ("plain", "trilinear", 24),
                                           ("hutchinson", "nearest", 24),
                                           ("fixed", "trilinear", 24),
                                           ("hutchinson", "trilinear", 26),
                                           ("hutchinson", "trilinear", 4),
                                           ("hutchinson", "trilinear", 6),
                                           ("fixed", "trilinear", 10)])
def test_precond_sgd_steps_follow_oracle(h, mode, interp, M):
    """Three iterations of Algorithm 1 on consecutive mini-batches: the same
    eta choices as the literal oracle loop and iterates within tolerance
    (M = 26: x rows of a length that is not a multiple of 4; M = 4, 6, 10:
    the smallest grids, where the element-wise kernels' 2 x 2 voxel blocks and
    32-byte chunks meet the grid's edges on every side)."""
    from paper_2311_16100_gb300.ops import SGDState
    B, nb = 12, 3
    c = Case(M, B * nb, interp=interp, ctf=True, seed=29)
    g = c.to_gpu()
    geom = c.gpu_geometry()
    lam, scale, beta, carm, K, seed = 1e-2, float(nb), 0.9, 0.5, 8, 31
    alpha = O.alpha_threshold(c.df, M, c.r_max, c.ctf, lam)
    v0 = (0.3 * c.vol).astype(np.complex64)
    D0 = np.ones((M, M, M))
    if mode == "fixed":
        D0 = O.exact_diag(c.R, c.df, lam=lam, scale=1.0, **c.geo()).astype(np.float32)
    st = SGDState(torch.from_numpy(v0).cuda(), mode=mode, alpha=alpha, eta0=4.0, beta=beta,
                  armijo_c=carm, n_probes=K, seed=seed,
                  D=torch.from_numpy(np.asarray(D0, np.float32)).cuda())
    ov, oD, oDa, oeta = v0.astype(np.complex128), np.asarray(D0, np.float64), np.zeros((M, M, M)), 4.0
    for k in range(1, nb + 1):
        sl = slice((k - 1) * B, k * B)
        h.precond_sgd_step(geom, st, g["images"][sl].contiguous(), g["rot"][sl].contiguous(),
                           g["df"][sl].contiguous(), lam, scale)
        out = O.alg1_step(ov, oD, oDa, oeta, k, c.images[sl], c.R[sl], c.df[sl], lam=lam,
                          scale=scale, alpha=alpha, beta=beta, c=carm, mode=mode, n_probes=K,
                          seed=seed, **c.geo())
        sc = cpu(st.scalars)
        assert sc[6] == out["halvings"] and sc[0] == out["eta"]
        assert abs(sc[3] - out["loss"]) <= 1e-5 * abs(out["loss"])
        assert rel_l2(cpu(st.v), out["v"]) <= TOL_GRAD
        if mode == "hutchinson":
            assert rel_l2(cpu(st.D), out["D"]) <= TOL_GRAD
        ov, oD, oDa, oeta = out["v"], out["D"], out["D_avg"], out["eta"]
        assert sc[1] == k


def test_rel_err(h):
    c = Case(32, 1, seed=37)
    a = c.vol
    b = (c.vol + 0.05 * O.ball_mask(32, 15).reshape(32, 32, 32)).astype(np.complex64)
    e = float(h.rel_err(c.gpu_geometry(), torch.from_numpy(b).cuda(), torch.from_numpy(a).cuda()))
    # FP32 differences against FP64 ones: a few float ulps of relative error
    assert abs(e - O.rel_err(b, a, 32, 15)) <= 2e-5 * e


def test_cells_outside_the_grid(h, request):
    """A scaled rotation sends outer pixels' cells past the grid edge: those
    corners contribute nothing (both sides), exercising the guarded paths."""
    if h.algo_name == "tiled":
        pytest.skip("the tiled algorithm bins with orthonormal rotations")
    c = Case(32, 9, interp="trilinear", ctf=True, seed=41)
    R = (1.08 * c.R).astype(np.float32)
    g = c.to_gpu()
    Rg = torch.from_numpy(R).cuda()
    geom = c.gpu_geometry()
    y = cpu(h.slice_project(geom, g["vol"], Rg, g["df"]))
    assert rel_l2(y, O.slice_project(c.vol, R, c.df, **c.geo())) <= TOL_SLICE
    loss, grad = h.loss_grad(geom, g["vol"], g["images"], Rg, g["df"], 0.1, 2.0)
    f, gw = O.loss_grad(c.vol, c.images, R, c.df, lam=0.1, scale=2.0, **c.geo())
    assert rel_l2(cpu(grad), gw) <= TOL_GRAD and abs(float(loss) - f) <= 1e-6 * abs(f)
    d = cpu(h.hutchinson_diag(geom, Rg, g["df"], 0.1, 2.0, n_probes=8, seed=3, probe_block=2))
    dw = O.hutchinson_diag(R, c.df, lam=0.1, scale=2.0, n_probes=8, seed=3, block=2, **c.geo())
    assert rel_l2(d, dw) <= TOL_GRAD


# ------------------------------------------------------------ validation
def test_invalid_arguments_are_rejected(h):
    from paper_2311_16100_gb300.ops import CryoSGDError, Geometry
    from paper_2311_16100_gb300 import native as N
    v = torch.zeros((16, 16, 16), dtype=torch.complex64, device="cuda")
    rot = torch.eye(3, device="cuda").reshape(1, 3, 3).contiguous()
    for geom, code in ((Geometry(15), N.CS_ERR_SHAPE), (Geometry(16, r_max=8), N.CS_ERR_SHAPE),
                       (Geometry(16, interp="cubic"), N.CS_ERR_ARG)):
        with pytest.raises(CryoSGDError) as e:
            h.slice_project(geom, v, rot, out=torch.empty((1, 16, 16), dtype=torch.complex64,
                                                          device="cuda"))
        assert e.value.status == code
    with pytest.raises(CryoSGDError):
        h.hutchinson_diag(Geometry(16), rot, n_probes=33)
    with pytest.raises(CryoSGDError):
        h.hvp(Geometry(16), torch.zeros((16, 16, 16), device="cuda"), rot, out=None,
              lam=float("nan"))


# ------------------------------------------------------- full-size launch
def test_loss_grad_full_size_m128_b1024(h):
    """The launch configuration of the benchmark (M = 128, trilinear, CTF,
    batch 1024), against the oracle on the whole batch."""
    c = Case(128, 1024, interp="trilinear", ctf=True, seed=3000)
    g = c.to_gpu()
    lam, scale = 1e-3, 50000 / 1024
    loss, grad = h.loss_grad(c.gpu_geometry(), g["vol"], g["images"], g["rot"], g["df"], lam, scale)
    f, gw = O.loss_grad(c.vol, c.images, c.R, c.df, lam=lam, scale=scale, **c.geo())
    assert rel_l2(cpu(grad), gw) <= TOL_GRAD
    assert abs(float(loss) - f) <= 1e-6 * abs(f)
