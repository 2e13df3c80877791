"""Steps fed from host memory (cs_precond_sgd_step_host): direct reads from
mapped pinned memory and double-buffered staging on the handle's copy stream
must give the same iterates as steps on device-resident batches, and the
loss read back into host memory."""
import numpy as np
import pytest

from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_state(ops, c, alpha):
    v0 = torch.from_numpy((0.3 * c.vol).astype(np.complex64)).cuda()
    return ops.SGDState(v0, mode="hutchinson", alpha=alpha, eta0=1.0, beta=0.9, armijo_c=0.5,
                        n_probes=8, seed=5)


@pytest.mark.parametrize("pinned,mode", [(True, "direct"), (True, "staged"), (False, "direct")])
def test_host_steps_match_device_steps(pinned, mode):
    """pinned + direct: the traversal reads the images from host memory;
    pinned + staged, and pageable memory in either mode: staged copies."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    B, nb = 16, 3
    c = Case(32, B * nb, interp="trilinear", ctf=True, seed=81)
    geom = c.gpu_geometry()
    h_dev, h_host = ops.Handle(0), ops.Handle(0)
    h_host.set_host_mode(mode)
    g = c.to_gpu()
    alpha = float(h_dev.threshold_alpha(geom, g["df"], B * nb, 0.01))
    st_dev, st_host = make_state(ops, c, alpha), make_state(ops, c, alpha)
    img = torch.from_numpy(c.images)
    q = torch.from_numpy(c.quat.astype(np.float32))
    df = torch.from_numpy(c.df)
    if pinned:
        img, q, df = img.pin_memory(), q.pin_memory(), df.pin_memory()
    losses = torch.zeros(6, dtype=torch.float64)
    if pinned:
        losses = losses.pin_memory()
    rot = torch.empty((B, 3, 3), device="cuda")
    dev_losses = []
    for k in range(6):
        sl = slice((k % nb) * B, (k % nb + 1) * B)
        h_host.precond_sgd_step_host(geom, st_host, img[sl], q[sl], df[sl], 0.01, float(nb),
                                     loss_host=losses[k])
        h_dev.quat_to_rot(g["quat"][sl].contiguous(), rot)
        h_dev.precond_sgd_step(geom, st_dev, g["images"][sl].contiguous(), rot,
                               g["df"][sl].contiguous(), 0.01, float(nb))
        dev_losses.append(st_dev.scalars[3].clone())
    torch.cuda.synchronize()
    assert rel_l2(st_host.v.cpu().numpy(), st_dev.v.cpu().numpy()) <= 1e-6
    assert float(st_host.scalars[0]) == float(st_dev.scalars[0])
    for k in range(6):
        assert abs(float(losses[k]) - float(dev_losses[k])) <= 1e-6 * abs(float(dev_losses[k]))
    h_dev.close()
    h_host.close()


def test_host_step_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    from paper_2311_16100_gb300.ops import CryoSGDError
    c = Case(16, 4, seed=83)
    h = ops.Handle(0)
    st = make_state(ops, c, 1.0)
    img = torch.from_numpy(c.images)
    q = torch.from_numpy(c.quat.astype(np.float32))
    with pytest.raises(CryoSGDError):          # CTF enabled, defocus missing
        h.precond_sgd_step_host(c.gpu_geometry(), st, img, q, None, 0.01, 1.0)
    with pytest.raises(ValueError):            # device tensor where host memory is required
        h.precond_sgd_step_host(c.gpu_geometry(), st, img.cuda(), q, None, 0.01, 1.0)
    with pytest.raises(KeyError):
        h.set_host_mode("zero-copy")
    with pytest.raises(CryoSGDError):
        h._check("cs_set_host_mode", h.lib.cs_set_host_mode(h.h, 7))
    h.close()


@pytest.mark.parametrize("algo", ["auto", "vector_slabs3", "pixel"])
def test_disc_packed_host_steps_match_device_steps(algo):
    """cs_precond_sgd_step_host_disc: the batch given as its disc pixels only
    (read where they land by the vector traversal, also split into z-slabs;
    spread into image layout first for the pixel algorithm) gives the same
    iterates as steps on the full images held on the device; r_max below
    M/2 - 1 and a batch size change between calls included."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops
    M, r = 32, 13
    sizes = (16, 16, 10, 16)
    c = Case(M, sum(sizes), interp="trilinear", ctf=True, seed=85, r_max=r)
    geom = c.gpu_geometry()
    h_dev, h_host = ops.Handle(0), ops.Handle(0)
    if algo == "vector_slabs3":
        h_host.set_algo("vector")
        h_host.set_slabs(3)
    else:
        h_host.set_algo(algo)
    g = c.to_gpu()
    alpha = float(h_dev.threshold_alpha(geom, g["df"], sum(sizes), 0.01))
    st_dev, st_host = make_state(ops, c, alpha), make_state(ops, c, alpha)
    disc = ops.pack_disc(torch.from_numpy(c.images), r).pin_memory()
    assert disc.shape == (sum(sizes), ops.disc_pixels(M, r))
    q = torch.from_numpy(c.quat.astype(np.float32)).pin_memory()
    df = torch.from_numpy(c.df).pin_memory()
    losses = torch.zeros(len(sizes), dtype=torch.float64).pin_memory()
    rot = torch.empty((max(sizes), 3, 3), device="cuda")
    start = 0
    dev_losses = []
    for k, B in enumerate(sizes):
        sl = slice(start, start + B)
        start += B
        h_host.precond_sgd_step_host_disc(geom, st_host, disc[sl], q[sl], df[sl], 0.01, 2.0,
                                          loss_host=losses[k])
        h_dev.quat_to_rot(g["quat"][sl].contiguous(), rot[:B])
        h_dev.precond_sgd_step(geom, st_dev, g["images"][sl].contiguous(), rot[:B],
                               g["df"][sl].contiguous(), 0.01, 2.0)
        dev_losses.append(st_dev.scalars[3].clone())
    torch.cuda.synchronize()
    assert rel_l2(st_host.v.cpu().numpy(), st_dev.v.cpu().numpy()) <= 1e-6
    assert float(st_host.scalars[0]) == float(st_dev.scalars[0])
    for k in range(len(sizes)):
        assert abs(float(losses[k]) - float(dev_losses[k])) <= 1e-6 * abs(float(dev_losses[k]))
    assert ops.disc_pixels(M, M // 2 - 1) == 709
    with pytest.raises(ValueError):
        ops.disc_pixels(M, M // 2)
    # a failed device-side range check (debug variant) would be reported here
    h_host.check_device_status()
    h_dev.close()
    h_host.close()


def test_disc_packed_host_steps_full_size():
    """The benchmark's end-to-end path at its size: 128^3, batches of 1024
    images given as their disc pixels in pinned host memory, trilinear + CTF,
    32 probes; two steps give the iterates of the same steps on the full
    images held on the device (inputs made on the device: a random volume,
    its slices plus noise)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops, synth
    M, r, B, nb, lam = 128, 63, 1024, 2, 0.01
    N = B * nb
    geom = ops.Geometry(M, r, "trilinear", ops.CTF())
    h_dev, h_host = ops.Handle(0), ops.Handle(0)
    vol = torch.from_numpy(synth.complex_normal((M, M, M), 91, 1.0).astype(np.complex64)).cuda()
    quat = torch.from_numpy(synth.shoemake_quaternions(N, 92).astype(np.float32))
    df = torch.from_numpy(synth.defocus_angstrom(N, 93).astype(np.float32))
    rot_all = h_dev.quat_to_rot(quat.cuda())
    images = h_dev.slice_project(geom, vol, rot_all, df.cuda())
    gen = torch.Generator(device="cuda").manual_seed(94)
    images = images + 0.3 * torch.complex(torch.randn(images.shape, generator=gen, device="cuda"),
                                          torch.randn(images.shape, generator=gen, device="cuda"))
    alpha = float(h_dev.threshold_alpha(geom, df.cuda(), N, lam))
    states = [ops.SGDState((0.3 * vol).contiguous(), mode="hutchinson", alpha=alpha, eta0=1.0,
                           beta=0.9, armijo_c=0.5, n_probes=32, seed=95) for _ in range(2)]
    st_dev, st_host = states
    disc = ops.pack_disc(images.cpu(), r).pin_memory()
    qh, dfh = quat.pin_memory(), df.pin_memory()
    losses = torch.zeros(nb, dtype=torch.float64).pin_memory()
    dev_losses = []
    for k in range(nb):
        sl = slice(k * B, (k + 1) * B)
        h_host.precond_sgd_step_host_disc(geom, st_host, disc[sl], qh[sl], dfh[sl], lam,
                                          float(nb), loss_host=losses[k])
        h_dev.precond_sgd_step(geom, st_dev, images[sl].contiguous(), rot_all[sl].contiguous(),
                               df[sl].cuda(), lam, float(nb))
        dev_losses.append(st_dev.scalars[3].clone())
    torch.cuda.synchronize()
    assert rel_l2(st_host.v.cpu().numpy(), st_dev.v.cpu().numpy()) <= 1e-6
    assert rel_l2(st_host.D.cpu().numpy(), st_dev.D.cpu().numpy()) <= 1e-6
    assert float(st_host.scalars[0]) == float(st_dev.scalars[0])
    for k in range(nb):
        assert abs(float(losses[k]) - float(dev_losses[k])) <= 1e-6 * abs(float(dev_losses[k]))
    h_host.check_device_status()
    h_dev.close()
    h_host.close()
