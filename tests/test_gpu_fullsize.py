"""The 256^3 workload at its full batch (1024 images of 256x256, the launch
configuration the benchmark times: vector traversal split into z-slabs,
tile-ordered table, per-slab item lists) against the pixel algorithm (one
scalar reduction per corner, one launch, row-ordered table), which the
parity suite checks against the FP64 oracle: the two must agree to FP32
summation-order differences.  The oracle itself is too slow at this size;
this is the "property at any size" check, plus the oracle on sampled
voxels of the exact diagonal under nearest interpolation (a count)."""
import numpy as np
import pytest

import oracle as O
from cryo_cases import rel_l2
from paper_2311_16100_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, B = 256, 1024


@pytest.fixture(scope="module")
def work():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    d = torch.device("cuda")
    h = ops.Handle(0)
    geom = ops.Geometry(M, M // 2 - 1, "trilinear", ops.CTF())
    vol = torch.from_numpy(synth.blob_volume(M, 5000, seed=5000)).to(d)
    q = torch.from_numpy(synth.shoemake_quaternions(B, 5001).astype(np.float32)).to(d)
    rot = h.quat_to_rot(q)
    df = torch.from_numpy(synth.defocus_angstrom(B, 5002).astype(np.float32)).to(d)
    images = h.slice_project(geom, vol, rot, df)
    gen = torch.Generator(device=d)
    gen.manual_seed(5003)
    images += 0.5 * torch.randn(images.shape, dtype=torch.complex64, device=d, generator=gen)
    v = (0.7 * vol).contiguous()
    yield ops, h, geom, v, images, rot, df, q
    h.close()


def handles(ops):
    hv, hp = ops.Handle(0), ops.Handle(0)
    hv.set_algo("vector")            # slab count from the grid's footprint (6 / 2 at 256^3)
    hp.set_algo("pixel")
    return hv, hp


def test_loss_grad_slabbed_vector_equals_pixel(work):
    ops, h, geom, v, images, rot, df, _ = work
    hv, hp = handles(ops)
    lv, gv = hv.loss_grad(geom, v, images, rot, df, 0.3, 100.0)
    lp, gp = hp.loss_grad(geom, v, images, rot, df, 0.3, 100.0)
    assert rel_l2(gv.cpu().numpy(), gp.cpu().numpy()) <= 1e-5
    assert abs(float(lv) - float(lp)) <= 1e-6 * abs(float(lp))
    hv.close()
    hp.close()


def test_hutchinson_slabbed_vector_equals_pixel(work):
    ops, h, geom, v, images, rot, df, _ = work
    hv, hp = handles(ops)
    dv = hv.hutchinson_diag(geom, rot, df, 0.3, 100.0, n_probes=32, seed=9, probe_block=4)
    dp = hp.hutchinson_diag(geom, rot, df, 0.3, 100.0, n_probes=32, seed=9, probe_block=4)
    assert rel_l2(dv.cpu().numpy(), dp.cpu().numpy()) <= 1e-5
    hv.close()
    hp.close()


def test_sgd_step_slabbed_vector_equals_pixel(work):
    ops, h, geom, v, images, rot, df, _ = work
    hv, hp = handles(ops)
    alpha = float(h.threshold_alpha(geom, df, 102400, 0.3))
    states = [ops.SGDState(v, mode="hutchinson", alpha=alpha, n_probes=32, seed=7)
              for _ in range(2)]
    for _ in range(2):
        hv.precond_sgd_step(geom, states[0], images, rot, df, 0.3, 100.0)
        hp.precond_sgd_step(geom, states[1], images, rot, df, 0.3, 100.0)
    assert float(states[0].scalars[0]) == float(states[1].scalars[0])      # same eta
    assert rel_l2(states[0].v.cpu().numpy(), states[1].v.cpu().numpy()) <= 1e-5
    assert rel_l2(states[0].D.cpu().numpy(), states[1].D.cpu().numpy()) <= 1e-5
    hv.close()
    hp.close()


def test_nearest_exact_diag_sampled_voxels_against_oracle(work):
    """Under nearest interpolation without CTF the diagonal is lam + the
    number of (image, pixel) pairs whose nearest voxel is j; the oracle's
    FP32 index rule gives each pixel's voxel, so sampled voxels are exact."""
    ops, h, _, _, _, rot, _, _ = work
    geom = ops.Geometry(M, M // 2 - 1, "nearest", None)
    n_img = 64
    d, _, _ = h.exact_diag(geom, rot[:n_img].contiguous(), None, 0.5, 1.0)
    d = d.cpu().numpy().ravel()
    R = rot[:n_img].cpu().numpy()
    count = np.zeros(M ** 3)
    for i in range(n_img):
        pix, vox, w = O.stencil(R[i], M, M // 2 - 1, "nearest")
        np.add.at(count, vox[:, 0][w[:, 0] > 0], 1.0)
    rng = np.random.default_rng(1)
    hit = np.flatnonzero(count)
    idx = np.concatenate([rng.choice(hit, 2000, replace=False),
                          rng.integers(0, M ** 3, 2000)])
    np.testing.assert_allclose(d[idx], count[idx] + 0.5, rtol=0, atol=1e-3)


def test_largest_grid_slices_and_gradient():
    """M = 512, the largest grid the library accepts: slices against the
    oracle, and the slab-split gradient (16 slabs) against the pixel
    algorithm (one launch, row-ordered table)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    Mx, Bx = 512, 3
    g = np.random.default_rng(512)
    vol = (g.normal(size=(Mx, Mx, Mx)).astype(np.float32)
           + 1j * g.normal(size=(Mx, Mx, Mx)).astype(np.float32)).astype(np.complex64)
    q = synth.shoemake_quaternions(Bx, 513)
    R = O.quat_to_rot(q).astype(np.float32)
    df = synth.defocus_angstrom(Bx, 514).astype(np.float32)
    d = torch.device("cuda")
    tv, tR, tdf = torch.from_numpy(vol).to(d), torch.from_numpy(R).to(d), torch.from_numpy(df).to(d)
    ctf = dict(kv=synth.CTF_KV, cs_mm=synth.CTF_CS_MM, amp=synth.CTF_AMP, pixel_A=synth.CTF_PIXEL_A)
    hv, hp = ops.Handle(0), ops.Handle(0)
    hv.set_algo("vector")
    hp.set_algo("pixel")
    for interp in ("nearest", "trilinear"):
        geom = ops.Geometry(Mx, Mx // 2 - 1, interp, ops.CTF())
        y = hv.slice_project(geom, tv, tR, tdf).cpu().numpy()
        want = O.slice_project(vol, R, df, Mx, Mx // 2 - 1, interp, ctf)
        assert rel_l2(y, want) <= 1e-5
    geom = ops.Geometry(Mx, Mx // 2 - 1, "trilinear", ops.CTF())
    images = torch.from_numpy((0.9 * want).astype(np.complex64)).to(d)
    del want
    lv, gv = hv.loss_grad(geom, tv, images, tR, tdf, 0.1, 10.0)
    lp, gp = hp.loss_grad(geom, tv, images, tR, tdf, 0.1, 10.0)
    assert rel_l2(gv.cpu().numpy(), gp.cpu().numpy()) <= 1e-5
    assert abs(float(lv) - float(lp)) <= 1e-6 * abs(float(lp))
    hv.close()
    hp.close()


@pytest.mark.parametrize("Mg", [160, 192])
def test_slab_policy_steps_match_one_slab(Mg):
    """At 160^3 the reduction pass runs in 2 z-slabs and the curvature as one
    pass over the tile-ordered table (skipping its holes); at 192^3 in 3
    slabs.  Three Algorithm-1 steps from the same state must match those of a
    handle with one slab (row-ordered table) up to summation order."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    Bg, nb = 96, 3
    d = torch.device("cuda")
    geom = ops.Geometry(Mg, Mg // 2 - 1, "trilinear", ops.CTF())
    h_def, h_one = ops.Handle(0), ops.Handle(0)
    h_one.set_slabs(1)
    vol = torch.from_numpy(synth.blob_volume(Mg, 400, seed=Mg)).to(d)
    q = torch.from_numpy(synth.shoemake_quaternions(Bg * nb, Mg + 1).astype(np.float32)).to(d)
    rot = h_def.quat_to_rot(q)
    df = torch.from_numpy(synth.defocus_angstrom(Bg * nb, Mg + 2).astype(np.float32)).to(d)
    images = h_def.slice_project(geom, vol, rot, df)
    alpha = float(h_def.threshold_alpha(geom, df, Bg * nb, 0.05))
    st = [ops.SGDState((0.5 * vol).contiguous(), mode="hutchinson", alpha=alpha, eta0=1.0,
                       n_probes=16, seed=3) for _ in range(2)]
    for k in range(nb):
        sl = slice(k * Bg, (k + 1) * Bg)
        for h, s in ((h_def, st[0]), (h_one, st[1])):
            h.precond_sgd_step(geom, s, images[sl].contiguous(), rot[sl].contiguous(),
                               df[sl].contiguous(), 0.05, float(nb))
    torch.cuda.synchronize()
    a, b = st[0].scalars.cpu().numpy(), st[1].scalars.cpu().numpy()
    assert a[0] == b[0]                                   # same step sizes
    assert abs(a[3] - b[3]) <= 1e-6 * abs(b[3])           # batch loss
    assert rel_l2(st[0].v.cpu().numpy(), st[1].v.cpu().numpy()) <= 1e-5
    assert rel_l2(st[0].D.cpu().numpy(), st[1].D.cpu().numpy()) <= 1e-5
    h_def.close()
    h_one.close()
