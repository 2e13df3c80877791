"""The C ABI library loads and exports every symbol include/cryosgd.h
declares, and the ctypes structure layouts match the C compiler's (no GPU
needed; no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cryosgd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_16100_gb300 import build, native
    build.build()
    return native.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_ctypes_signatures_cover_the_header():
    from paper_2311_16100_gb300 import native
    assert set(native.SIGNATURES) == set(declared_functions())


def test_status_strings(lib):
    from paper_2311_16100_gb300 import native as N
    for code, name in ((N.CS_OK, b"CS_OK"), (N.CS_ERR_SHAPE, b"CS_ERR_SHAPE"),
                       (N.CS_ERR_ALLOC, b"CS_ERR_ALLOC")):
        assert lib.cs_status_string(code) == name


def test_null_handle_is_an_argument_error(lib):
    from paper_2311_16100_gb300 import native as N
    assert lib.cs_slice_project(None, None, None, None, None, 0, None, None) == N.CS_ERR_ARG
    assert lib.cs_destroy(None) == N.CS_OK
    assert lib.cs_last_error(None) == b""


def test_struct_layouts_match_c(tmp_path):
    from paper_2311_16100_gb300 import native as N
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "cryosgd.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(cs_ctf), sizeof(cs_geom), offsetof(cs_geom, ctf),
         offsetof(cs_ctf, enabled));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(cs_sgd_state), offsetof(cs_sgd_state, scalars),
         offsetof(cs_sgd_state, seed), offsetof(cs_sgd_state, beta),
         offsetof(cs_sgd_state, c), offsetof(cs_sgd_state, max_halvings));
  printf("%d %d %d\n", CS_NSCALARS, CS_S_HALVINGS, CS_MAX_M);
  printf("%zu %zu %zu %zu %zu\n", sizeof(cs_problem), offsetof(cs_problem, state),
         offsetof(cs_problem, images), offsetof(cs_problem, B), offsetof(cs_problem, scale));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = list(map(int, out))
    want = [ctypes.sizeof(N.CsCtf), ctypes.sizeof(N.CsGeom), N.CsGeom.ctf.offset,
            N.CsCtf.enabled.offset,
            ctypes.sizeof(N.CsSgdState), N.CsSgdState.scalars.offset, N.CsSgdState.seed.offset,
            N.CsSgdState.beta.offset, N.CsSgdState.c.offset, N.CsSgdState.max_halvings.offset,
            N.CS_NSCALARS, N.CS_S_HALVINGS, N.CS_MAX_M,
            ctypes.sizeof(N.CsProblem), N.CsProblem.state.offset, N.CsProblem.images.offset,
            N.CsProblem.B.offset, N.CsProblem.scale.offset]
    assert got == want


def test_product_path_fails_loudly_without_library(monkeypatch):
    from paper_2311_16100_gb300 import native
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", "/nonexistent/libcryosgd.so")
    with pytest.raises(ImportError):
        native.load()
