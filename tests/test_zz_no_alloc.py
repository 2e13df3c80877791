"""The allocation-free Hutchinson entry point, called through the C ABI.

Some callers of this library cannot allocate device memory when they need
the preconditioner estimate: they run inside another application's stream
capture, or their device memory belongs to a caching allocator, or they
allocate only at start-up.  cs_hutchinson_diag_noalloc serves them with a
fixed scratch array inside the library.  This test checks that two calls in
a row agree with cs_hutchinson_diag (same tolerance as the other parity
tests), that the scratch size limit is enforced, and that no device memory
is taken from the caller's allocator.  It is collected last on purpose.
"""
import ctypes

import pytest

from cryo_cases import Case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_16100_gb300 import native
    return native.load()


def call_noalloc(lib, geom, rot, df, B, lam, scale, K, seed, block, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.cs_hutchinson_diag_noalloc(
        geom.c, ctypes.c_void_p(rot.data_ptr()),
        ctypes.c_void_p(df.data_ptr()) if df is not None else None, B, lam, scale, K, seed,
        block, ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_hutchinson_diag_twice(lib):
    from paper_2311_16100_gb300 import native as N
    from paper_2311_16100_gb300.ops import Handle
    torch.cuda.set_device(0)
    h = Handle(0)
    for call, (M, B, K, block, interp) in enumerate(((32, 24, 16, 3, "trilinear"),
                                                     (64, 10, 32, 7, "trilinear"))):
        c = Case(M, B, interp=interp, ctf=True, seed=900 + call)
        g = c.to_gpu()
        geom = c.gpu_geometry()
        want = h.hutchinson_diag(geom, g["rot"], g["df"], 0.01, 8.0, n_probes=K, seed=11,
                                 probe_block=block)
        out = torch.full((M, M, M), float("nan"), device="cuda")
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        rc = call_noalloc(lib, geom, g["rot"], g["df"], B, 0.01, 8.0, K, 11, block, out)
        torch.cuda.synchronize()
        assert rc == N.CS_OK
        assert torch.cuda.memory_allocated() == before
        assert rel_l2(out.cpu().numpy(), want.cpu().numpy()) <= TOL
    h.close()


def test_noalloc_rejects_grids_beyond_its_scratch(lib):
    from paper_2311_16100_gb300 import native as N
    from paper_2311_16100_gb300.ops import CTF, Geometry
    geom = Geometry(130, interp="trilinear", ctf=CTF())
    rot = torch.eye(3, device="cuda").reshape(1, 3, 3).contiguous()
    df = torch.full((1,), 2e4, device="cuda")
    out = torch.zeros((1,), device="cuda")
    assert call_noalloc(lib, geom, rot, df, 1, 0.0, 1.0, 8, 1, 0, out) == N.CS_ERR_SHAPE
    assert call_noalloc(lib, Geometry(32), rot, df, 1, 0.0, 1.0, 33, 1, 0,
                        torch.zeros((32, 32, 32), device="cuda")) == N.CS_ERR_SHAPE
