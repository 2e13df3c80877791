"""Failure handling without a GPU fault: a bounded device-side wait that
runs out is reported through the status word (and the context stays
usable), and a workspace allocation failure (injected on the host) is
reported as CS_ERR_ALLOC and leaves the handle usable."""
import os

import pytest

import oracle as O
from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import ops as o
    return o


def test_bounded_wait_expiry_is_reported_and_cleared(ops):
    from paper_2311_16100_gb300 import native as N
    h = ops.Handle(0)
    h.check_device_status()                        # clean to begin with
    h.selftest_wait_timeout(2000)
    with pytest.raises(ops.CryoSGDError) as e:
        h.check_device_status()
    assert e.value.status == N.CS_ERR_TIMEOUT
    h.check_device_status()                        # the report clears the word
    c = Case(24, 5, interp="trilinear", ctf=True, seed=91)
    g = c.to_gpu()
    y = h.slice_project(c.gpu_geometry(), g["vol"], g["rot"], g["df"]).cpu().numpy()
    assert rel_l2(y, O.slice_project(c.vol, c.R, c.df, **c.geo())) <= 1e-5
    with pytest.raises(ops.CryoSGDError):
        h.selftest_wait_timeout(0)
    h.close()


def test_workspace_allocation_failure_is_reported(ops):
    from paper_2311_16100_gb300 import native as N
    h = ops.Handle(0)
    c = Case(24, 6, interp="trilinear", ctf=True, seed=92)
    g = c.to_gpu()
    os.environ["CS_FAULT_INJECT_ALLOC"] = "1"
    try:
        with pytest.raises(ops.CryoSGDError) as e:
            h.loss_grad(c.gpu_geometry(), g["vol"], g["images"], g["rot"], g["df"], 0.1, 2.0)
        assert e.value.status == N.CS_ERR_ALLOC
    finally:
        del os.environ["CS_FAULT_INJECT_ALLOC"]
    loss, grad = h.loss_grad(c.gpu_geometry(), g["vol"], g["images"], g["rot"], g["df"], 0.1, 2.0)
    f, gw = O.loss_grad(c.vol, c.images, c.R, c.df, lam=0.1, scale=2.0, **c.geo())
    assert rel_l2(grad.cpu().numpy(), gw) <= 1e-4
    h.close()
