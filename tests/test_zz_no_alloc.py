"""The allocation-free Hutchinson entry point, called through the C ABI.

Some callers of this library cannot allocate device memory when they need
the preconditioner estimate: they run inside another application's stream
capture, or their device memory belongs to a caching allocator, or they
allocate only at start-up.  cs_hutchinson_diag_noalloc serves them with a
fixed scratch array inside the library.  This test checks that calls in a
row agree with cs_hutchinson_diag (same tolerance as the other parity
tests) under trilinear and nearest interpolation, up to the largest grid the
scratch holds (128^3) and for an empty batch, that the size limit and the
argument checks are enforced, and that the calls take no device memory,
neither from the caller's allocator nor from the device (cudaMemGetInfo).
It is collected last on purpose.
"""
import ctypes
import gc

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


# (M, B, probes, probe block, interpolation, CTF)
CASES = ((32, 24, 16, 3, "trilinear", True),
         (64, 10, 32, 7, "trilinear", True),
         (128, 4, 32, 2, "trilinear", True),      # the largest grid the scratch holds
         (32, 20, 8, 5, "nearest", False),
         (40, 16, 1, 9, "nearest", True),
         (16, 0, 32, 1, "trilinear", True))       # empty batch: diag = lambda


def test_noalloc_matches_hutchinson_diag_in_a_row(lib):
    from paper_2311_16100_gb300 import native as N
    from paper_2311_16100_gb300.ops import Handle
    torch.cuda.set_device(0)
    h = Handle(0)
    lam, scale = 0.01, 8.0
    for call, (M, B, K, block, interp, ctf) in enumerate(CASES):
        c = Case(M, max(B, 1), interp=interp, ctf=ctf, seed=900 + call)
        g = c.to_gpu()
        geom = c.gpu_geometry()
        # with B = 0 the pointers stay valid, and the call must not read them
        rot = g["rot"]
        df = g["df"] if ctf else None
        want = h.hutchinson_diag(geom, rot[:B].contiguous(),
                                 df[:B].contiguous() if ctf else None, lam, scale,
                                 n_probes=K, seed=11, probe_block=block)
        outs = []
        for rep in range(2):                     # two calls in a row on the shared scratch
            out = torch.full((M, M, M), float("nan"), device="cuda")
            torch.cuda.synchronize()
            # no garbage collection inside the measured window: freeing an
            # earlier test's tensors there would change the counters
            gc.collect()
            gc.disable()
            try:
                before = torch.cuda.memory_allocated()
                free_before = torch.cuda.mem_get_info()[0]
                rc = call_noalloc(lib, geom, rot, df, B, lam, scale, K, 11, block, out)
                torch.cuda.synchronize()
                free_after = torch.cuda.mem_get_info()[0]
                after = torch.cuda.memory_allocated()
            finally:
                gc.enable()
            assert rc == N.CS_OK, (M, B, interp, rep)
            assert after == before
            if call > 0 or rep > 0:
                # after the first call (which may load the library's kernels)
                # no device memory changes hands
                assert free_after == free_before, (M, B, interp, rep)
            outs.append(out)
        for out in outs:
            if B == 0:
                assert bool(torch.all(out == lam)) and bool(torch.all(want == lam))
            else:
                assert rel_l2(out.cpu().numpy(), want.cpu().numpy()) <= TOL, (M, B, interp)
    h.close()


def test_noalloc_rejects_bad_arguments(lib):
    from paper_2311_16100_gb300 import native as N
    from paper_2311_16100_gb300.ops import CTF, Geometry
    rot = torch.eye(3, device="cuda").reshape(1, 3, 3).contiguous()
    df = torch.full((1,), 2e4, device="cuda")
    out = torch.zeros((1,), device="cuda")
    geom = Geometry(130, interp="trilinear", ctf=CTF())       # beyond the fixed scratch
    assert call_noalloc(lib, geom, rot, df, 1, 0.0, 1.0, 8, 1, 0, out) == N.CS_ERR_SHAPE
    small = torch.zeros((32, 32, 32), device="cuda")
    assert call_noalloc(lib, Geometry(32), rot, df, 1, 0.0, 1.0, 33, 1, 0,
                        small) == N.CS_ERR_SHAPE
    for bad in (CTF(kv=float("inf")), CTF(pixel_A=float("inf")), CTF(cs_mm=float("inf")),
                CTF(kv=float("nan")), CTF(amp=1.0)):
        assert call_noalloc(lib, Geometry(32, ctf=bad), rot, df, 1, 0.0, 1.0, 8, 1, 0,
                            small) == N.CS_ERR_ARG
    assert call_noalloc(lib, Geometry(32), rot, df, 1, float("inf"), 1.0, 8, 1, 0,
                        small) == N.CS_ERR_ARG
    torch.cuda.synchronize()
    assert bool(torch.all(small == 0))           # nothing was enqueued
