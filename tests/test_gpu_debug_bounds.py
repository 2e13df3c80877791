"""The parity suite under the debug variant of the library.

libcryosgd_debug.so (built by build() with -DCS_DEBUG_BOUNDS) range-checks
every gather and scatter index of the traversal kernels on the device: an
index out of range skips its access and cs_check_device_status reports
CS_ERR_INTERNAL.  This runs the small parity cases (every scatter algorithm,
the three-slab traversal) and the host-fed steps (whole and disc-packed
images) in a child process that loads that variant (CS_LIBRARY=debug); each
handle's status is checked when its tests end, so any failed range check
fails the run.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_loaded_library_variant():
    """The library this process loaded is the variant CS_LIBRARY asks for."""
    from paper_2311_16100_gb300 import native
    lib = native.load()
    want = native.CS_BUILD_DEBUG_BOUNDS if os.environ.get("CS_LIBRARY") == "debug" else 0
    assert lib.cs_build_flags() == want


def test_parity_suite_under_range_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(os.path.join(ROOT, "paper_2311_16100_gb300", "libcryosgd_debug.so")):
        pytest.fail("libcryosgd_debug.so is not built (run build())")
    env = dict(os.environ, CS_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "gpu", "tests/test_gpu_parity.py",
                        "tests/test_gpu_host_step.py",
                        "tests/test_gpu_debug_bounds.py::test_loaded_library_variant",
                        "-k", "not full_size"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
