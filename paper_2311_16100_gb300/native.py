"""ctypes declarations of libcryosgd's C ABI (include/cryosgd.h).

Loading fails loudly when the in-tree library has not been built: there is
no CPU fallback.  Build it with ``python -m paper_2311_16100_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_longlong, POINTER, c_char_p, c_double, c_float, c_int, c_size_t, c_uint64, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
# CS_LIBRARY=debug selects the debug variant (device-side index range
# checks, reported by cs_check_device_status)
LIB_PATH = os.path.join(PKG, "libcryosgd_debug.so" if os.environ.get("CS_LIBRARY") == "debug"
                        else "libcryosgd.so")
CS_BUILD_DEBUG_BOUNDS = 1

CS_OK, CS_ERR_ARG, CS_ERR_SHAPE, CS_ERR_CUDA, CS_ERR_TIMEOUT, CS_ERR_INTERNAL, CS_ERR_ALLOC = range(7)
CS_NEAREST, CS_TRILINEAR = 0, 1
CS_PLAIN, CS_HUTCHINSON, CS_FIXED = 0, 1, 2
CS_ALGO_AUTO, CS_ALGO_PIXEL, CS_ALGO_TILED, CS_ALGO_VECTOR = 0, 1, 2, 3
CS_HOST_STAGED, CS_HOST_DIRECT = 0, 1
(CS_S_ETA, CS_S_K, CS_S_ALPHA, CS_S_LOSS, CS_S_G, CS_S_Q, CS_S_HALVINGS,
 CS_S_STATUS, CS_NSCALARS) = range(9)
CS_MAX_M = 512
(CS_PH_PRECOND, CS_PH_LOSS_GRAD, CS_PH_DIRECTION, CS_PH_CURVATURE, CS_PH_UPDATE,
 CS_NPHASES) = range(6)
PHASE_NAMES = ("precond", "loss_grad", "direction", "curvature", "update")


class CsCtf(ctypes.Structure):
    _fields_ = [("kv", c_float), ("cs_mm", c_float), ("amp", c_float),
                ("pixel_A", c_float), ("enabled", c_int)]


class CsGeom(ctypes.Structure):
    _fields_ = [("M", c_int), ("r_max", c_int), ("interp", c_int), ("ctf", CsCtf)]


class CsSgdState(ctypes.Structure):
    _fields_ = [("v", c_void_p), ("D", c_void_p), ("D_avg", c_void_p),
                ("scalars", c_void_p), ("mode", c_int), ("n_probes", c_int),
                ("seed", c_uint64), ("beta", c_float), ("c", c_float),
                ("max_halvings", c_int)]


class CsProblem(ctypes.Structure):
    _fields_ = [("geom", CsGeom), ("state", CsSgdState), ("images", c_void_p),
                ("quat", c_void_p), ("defocus", c_void_p), ("B", c_int), ("n_batches", c_int),
                ("lam", c_float), ("scale", c_float)]


CS_MAX_PROBLEMS = 8
CS_MLP_NPARAMS = 4481

P = c_void_p
G = POINTER(CsGeom)

# name -> (restype, argtypes)
SIGNATURES = {
    "cs_create": (c_int, [POINTER(c_void_p), c_int]),
    "cs_destroy": (c_int, [P]),
    "cs_last_error": (c_char_p, [P]),
    "cs_status_string": (c_char_p, [c_int]),
    "cs_reserve": (c_int, [P, c_int, c_int]),
    "cs_workspace_bytes": (c_size_t, [P]),
    "cs_set_algo": (c_int, [P, c_int]),
    "cs_quat_to_rot": (c_int, [P, P, c_int, P, P]),
    "cs_slice_project": (c_int, [P, G, P, P, P, c_int, P, P]),
    "cs_backproject_adjoint": (c_int, [P, G, P, P, P, c_int, c_float, P, P]),
    "cs_loss_grad": (c_int, [P, G, P, P, P, P, c_int, c_float, c_float, P, P, P]),
    "cs_hvp": (c_int, [P, G, P, P, P, c_int, c_float, c_float, P, P]),
    "cs_hutchinson_diag": (c_int, [P, G, P, P, c_int, c_float, c_float, c_int, c_uint64,
                                   c_uint64, P, P]),
    "cs_hutchinson_diag_noalloc": (c_int, [G, P, P, c_int, c_float, c_float, c_int, c_uint64,
                                           c_uint64, P, P]),
    "cs_precompute_preconditioner": (c_int, [P, G, P, P, c_int, c_int, c_int, c_float, c_int,
                                             c_uint64, P, P]),
    "cs_phase_shift": (c_int, [P, c_int, P, P, c_int, c_int, P]),
    "cs_set_slabs": (c_int, [P, c_int]),
    "cs_set_host_mode": (c_int, [P, c_int]),
    "cs_selftest_wait_timeout": (c_int, [P, c_longlong, P]),
    "cs_fsc": (c_int, [P, c_int, P, P, c_int, P, P, P]),
    "cs_shell_minmax": (c_int, [P, c_int, P, c_int, P, P, P, P]),
    "cs_exact_diag": (c_int, [P, G, P, P, c_int, c_float, c_float, P, P, P, P]),
    "cs_threshold_alpha": (c_int, [P, G, P, c_int, c_double, c_double, P, P]),
    "cs_precond_sgd_step": (c_int, [P, G, POINTER(CsSgdState), P, P, P, c_int, c_float,
                                    c_float, P]),
    "cs_precond_sgd_step_host": (c_int, [P, G, POINTER(CsSgdState), P, P, P, c_int, c_float,
                                         c_float, P, P]),
    "cs_precond_sgd_step_host_disc": (c_int, [P, G, POINTER(CsSgdState), P, P, P, c_int,
                                              c_float, c_float, P, P]),
    "cs_disc_pixels": (c_int, [c_int, c_int]),
    "cs_rel_err": (c_int, [P, G, P, P, P, P]),
    "cs_profile_enable": (c_int, [P, c_int, c_int]),
    "cs_profile_read": (c_int, [P, POINTER(c_double), POINTER(c_int)]),
    "cs_kernel_launches": (c_uint64, []),
    "cs_measure_reduction_rate": (c_int, [P, POINTER(c_double)]),
    "cs_multi_step": (c_int, [P, POINTER(CsProblem), c_int, P]),
    "cs_multi_step_graph": (c_int, [P, POINTER(CsProblem), c_int, POINTER(c_void_p)]),
    "cs_graph_launch": (c_int, [P, P]),
    "cs_graph_destroy": (c_int, [P]),
    "cs_set_launch_shape": (c_int, [P, c_int, c_int]),
    "cs_autotune": (c_int, [P, POINTER(CsProblem), c_int, POINTER(c_int), POINTER(c_int)]),
    "cs_mlp_forward": (c_int, [P, c_int, P, P, P, P, c_int, c_float, c_int, P]),
    "cs_mlp_grad": (c_int, [P, c_int, c_int, P, P, P, P, P, P, c_int, P]),
    "cs_mlp_adam_step": (c_int, [P, P, P, P, P, c_float, c_int, c_float, c_float, c_float,
                                 c_float, P]),
    "cs_mlp_target": (c_int, [P, c_int, c_int, P, c_float, P, P]),
    "cs_check_device_status": (c_int, [P]),
    "cs_build_flags": (c_int, []),
}

_lib = None


def load() -> ctypes.CDLL:
    """The loaded library, with argument types declared (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run "
            "`python -m paper_2311_16100_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
