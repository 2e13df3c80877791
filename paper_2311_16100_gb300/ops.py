"""Thin Python binding of libcryosgd: same names as the C ABI, argument
marshalling only.  Tensors are CUDA tensors owned by the caller (complex64
volumes / images, float32 rotations, defocus and real volumes, float64
scalars); every computation runs in the library's kernels on the current
torch CUDA stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import torch

from . import native as N


class CryoSGDError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} -> {status_string(status)}: {msg}")
        self.status = status


def kernel_launches() -> int:
    """Kernels launched by libcryosgd in this process so far."""
    return int(N.load().cs_kernel_launches())


def status_string(code: int) -> str:
    return N.load().cs_status_string(code).decode()


@dataclass
class CTF:
    """Microscope parameters of the CTF (kV, Cs in mm, amplitude contrast,
    pixel size in Angstrom)."""
    kv: float = 300.0
    cs_mm: float = 2.7
    amp: float = 0.1
    pixel_A: float = 1.5


@dataclass
class Geometry:
    """Grid side M, disc radius r_max (default M/2-1), interpolation
    ("nearest" | "trilinear") and an optional CTF."""
    M: int
    r_max: int | None = None
    interp: str = "trilinear"
    ctf: CTF | None = None
    _c: N.CsGeom = field(init=False, repr=False)

    def __post_init__(self):
        if self.r_max is None:
            self.r_max = self.M // 2 - 1
        c = N.CsGeom()
        c.M = self.M
        c.r_max = self.r_max
        c.interp = {"nearest": N.CS_NEAREST, "trilinear": N.CS_TRILINEAR}.get(self.interp, -1)
        if self.ctf is not None:
            c.ctf = N.CsCtf(self.ctf.kv, self.ctf.cs_mm, self.ctf.amp, self.ctf.pixel_A, 1)
        else:
            c.ctf = N.CsCtf(0, 0, 0, 0, 0)
        self._c = c

    @property
    def c(self):
        return ctypes.byref(self._c)


def _ptr(t: torch.Tensor | None, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t: torch.Tensor | None, dtype=None, name="tensor"):
    """Pointer of a host tensor (page-locked for asynchronous copies)."""
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError(f"{name} must be a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """Owns a cs_handle (device binding + workspace)."""

    def __init__(self, device: int | None = None):
        self.lib = N.load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.cs_create(ctypes.byref(h), device)
        if rc != N.CS_OK:
            raise CryoSGDError("cs_create", rc, "no usable CUDA device")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.cs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, fn: str, rc: int):
        if rc != N.CS_OK:
            raise CryoSGDError(fn, rc, self.lib.cs_last_error(self.h).decode())

    # ------------------------------------------------------------ calls
    def reserve(self, M: int, max_batch: int = 0):
        self._check("cs_reserve", self.lib.cs_reserve(self.h, M, max_batch))

    def set_algo(self, algo: str):
        """Scatter algorithm of the adjoint-type passes: "auto" (default),
        "vector", "pixel" or "tiled"."""
        code = {"auto": N.CS_ALGO_AUTO, "pixel": N.CS_ALGO_PIXEL, "tiled": N.CS_ALGO_TILED,
                "vector": N.CS_ALGO_VECTOR}[algo]
        self._check("cs_set_algo", self.lib.cs_set_algo(self.h, code))

    def workspace_bytes(self) -> int:
        return int(self.lib.cs_workspace_bytes(self.h))

    def quat_to_rot(self, quat, rot=None, stream=None):
        B = quat.shape[0]
        if rot is None:
            rot = torch.empty((B, 3, 3), dtype=torch.float32, device=quat.device)
        self._check("cs_quat_to_rot", self.lib.cs_quat_to_rot(
            self.h, _ptr(quat, torch.float32, "quat"), B, _ptr(rot, torch.float32, "rot"),
            _stream(stream)))
        return rot

    def slice_project(self, geom: Geometry, vol, rot, defocus=None, out=None, stream=None):
        B = rot.shape[0]
        M = geom.M
        if out is None:
            out = torch.empty((B, M, M), dtype=torch.complex64, device=vol.device)
        self._check("cs_slice_project", self.lib.cs_slice_project(
            self.h, geom.c, _ptr(vol, torch.complex64, "vol"), _ptr(rot, torch.float32, "rot"),
            _ptr(defocus, torch.float32, "defocus"), B, _ptr(out, torch.complex64, "out"),
            _stream(stream)))
        return out

    def backproject_adjoint(self, geom: Geometry, images, rot, defocus=None, scale=1.0,
                            vol_accum=None, stream=None):
        B = rot.shape[0]
        M = geom.M
        if vol_accum is None:
            vol_accum = torch.zeros((M, M, M), dtype=torch.complex64, device=images.device)
        self._check("cs_backproject_adjoint", self.lib.cs_backproject_adjoint(
            self.h, geom.c, _ptr(images, torch.complex64, "images"),
            _ptr(rot, torch.float32, "rot"), _ptr(defocus, torch.float32, "defocus"), B,
            float(scale), _ptr(vol_accum, torch.complex64, "vol_accum"), _stream(stream)))
        return vol_accum

    def loss_grad(self, geom: Geometry, vol, images, rot, defocus=None, lam=0.0, scale=1.0,
                  grad=None, loss=None, stream=None):
        B = rot.shape[0]
        if grad is None:
            grad = torch.empty_like(vol)
        if loss is None:
            loss = torch.empty((), dtype=torch.float64, device=vol.device)
        self._check("cs_loss_grad", self.lib.cs_loss_grad(
            self.h, geom.c, _ptr(vol, torch.complex64, "vol"),
            _ptr(images, torch.complex64, "images"), _ptr(rot, torch.float32, "rot"),
            _ptr(defocus, torch.float32, "defocus"), B, float(lam), float(scale),
            _ptr(grad, torch.complex64, "grad"), _ptr(loss, torch.float64, "loss"),
            _stream(stream)))
        return loss, grad

    def hvp(self, geom: Geometry, z, rot, defocus=None, lam=0.0, scale=1.0, out=None,
            stream=None):
        B = rot.shape[0]
        if out is None:
            out = torch.empty_like(z)
        self._check("cs_hvp", self.lib.cs_hvp(
            self.h, geom.c, _ptr(z, torch.float32, "z"), _ptr(rot, torch.float32, "rot"),
            _ptr(defocus, torch.float32, "defocus"), B, float(lam), float(scale),
            _ptr(out, torch.float32, "Hz"), _stream(stream)))
        return out

    def hutchinson_diag(self, geom: Geometry, rot, defocus=None, lam=0.0, scale=1.0,
                        n_probes=32, seed=0, probe_block=0, out=None, stream=None):
        B = rot.shape[0]
        M = geom.M
        if out is None:
            out = torch.empty((M, M, M), dtype=torch.float32, device=rot.device)
        self._check("cs_hutchinson_diag", self.lib.cs_hutchinson_diag(
            self.h, geom.c, _ptr(rot, torch.float32, "rot"),
            _ptr(defocus, torch.float32, "defocus"), B, float(lam), float(scale),
            int(n_probes), int(seed), int(probe_block), _ptr(out, torch.float32, "diag"),
            _stream(stream)))
        return out

    def precompute_preconditioner(self, geom: Geometry, rot_all, defocus_all=None, B=1024,
                                  n_epochs=1, lam=0.0, n_probes=32, seed=0, out=None,
                                  stream=None):
        N = rot_all.shape[0]
        M = geom.M
        if out is None:
            out = torch.empty((M, M, M), dtype=torch.float32, device=rot_all.device)
        self._check("cs_precompute_preconditioner", self.lib.cs_precompute_preconditioner(
            self.h, geom.c, _ptr(rot_all, torch.float32, "rot_all"),
            _ptr(defocus_all, torch.float32, "defocus_all"), N, int(B), int(n_epochs),
            float(lam), int(n_probes), int(seed), _ptr(out, torch.float32, "D_out"),
            _stream(stream)))
        return out

    def exact_diag(self, geom: Geometry, rot, defocus=None, lam=0.0, scale=1.0,
                   diag=True, coverage=False, ctf2w=False, stream=None):
        B = rot.shape[0]
        M = geom.M
        mk = lambda want: (torch.empty((M, M, M), dtype=torch.float32, device=rot.device)
                           if want is True else (want if want is not False else None))
        d, cv, cw = mk(diag), mk(coverage), mk(ctf2w)
        self._check("cs_exact_diag", self.lib.cs_exact_diag(
            self.h, geom.c, _ptr(rot, torch.float32, "rot"),
            _ptr(defocus, torch.float32, "defocus"), B, float(lam), float(scale),
            _ptr(d, torch.float32, "diag"), _ptr(cv, torch.float32, "coverage"),
            _ptr(cw, torch.float32, "ctf2w"), _stream(stream)))
        return d, cv, cw

    def threshold_alpha(self, geom: Geometry, defocus_all, N_images, lam, scale_alpha=1.0,
                        out=None, stream=None):
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=torch.device("cuda", self.device))
        self._check("cs_threshold_alpha", self.lib.cs_threshold_alpha(
            self.h, geom.c, _ptr(defocus_all, torch.float32, "defocus_all"), int(N_images),
            float(lam), float(scale_alpha), _ptr(out, torch.float64, "alpha"),
            _stream(stream)))
        return out

    def precond_sgd_step(self, geom: Geometry, state: "SGDState", images, rot, defocus=None,
                         lam=0.0, scale=1.0, stream=None):
        B = rot.shape[0]
        self._check("cs_precond_sgd_step", self.lib.cs_precond_sgd_step(
            self.h, geom.c, ctypes.byref(state.cstruct()), _ptr(images, torch.complex64, "images"),
            _ptr(rot, torch.float32, "rot"), _ptr(defocus, torch.float32, "defocus"), B,
            float(lam), float(scale), _stream(stream)))

    def precond_sgd_step_host(self, geom: Geometry, state: "SGDState", images_host, quat_host,
                              defocus_host=None, lam=0.0, scale=1.0, loss_host=None,
                              stream=None):
        """One step on a batch in (pinned) host memory; asynchronous: the
        host tensors and loss_host (a host float64 element) must not be
        touched until the stream has completed the step."""
        B = quat_host.shape[0]
        self._check("cs_precond_sgd_step_host", self.lib.cs_precond_sgd_step_host(
            self.h, geom.c, ctypes.byref(state.cstruct()),
            _hptr(images_host, torch.complex64, "images_host"),
            _hptr(quat_host, torch.float32, "quat_host"),
            _hptr(defocus_host, torch.float32, "defocus_host"), B, float(lam), float(scale),
            _hptr(loss_host, torch.float64, "loss_host"), _stream(stream)))

    def precond_sgd_step_host_disc(self, geom: Geometry, state: "SGDState", images_disc_host,
                                   quat_host, defocus_host=None, lam=0.0, scale=1.0,
                                   loss_host=None, stream=None):
        """As precond_sgd_step_host with images given as their disc pixels
        only, complex64 [B][n_px] (pack_disc); asynchronous likewise."""
        B = quat_host.shape[0]
        self._check("cs_precond_sgd_step_host_disc", self.lib.cs_precond_sgd_step_host_disc(
            self.h, geom.c, ctypes.byref(state.cstruct()),
            _hptr(images_disc_host, torch.complex64, "images_disc_host"),
            _hptr(quat_host, torch.float32, "quat_host"),
            _hptr(defocus_host, torch.float32, "defocus_host"), B, float(lam), float(scale),
            _hptr(loss_host, torch.float64, "loss_host"), _stream(stream)))

    def profile_enable(self, enable=True, max_steps=4096):
        self._check("cs_profile_enable", self.lib.cs_profile_enable(self.h, int(enable),
                                                                    int(max_steps)))

    def profile_read(self):
        """{phase: (total ms, timed steps)} of cs_precond_sgd_step."""
        ms = (ctypes.c_double * N.CS_NPHASES)()
        cnt = (ctypes.c_int * N.CS_NPHASES)()
        self._check("cs_profile_read", self.lib.cs_profile_read(self.h, ms, cnt))
        return {n: (ms[i], cnt[i]) for i, n in enumerate(N.PHASE_NAMES)}

    def measure_reduction_rate(self) -> float:
        """G 16-byte reductions per second into L2-resident memory (synchronous)."""
        g = ctypes.c_double()
        self._check("cs_measure_reduction_rate",
                    self.lib.cs_measure_reduction_rate(self.h, ctypes.byref(g)))
        return g.value

    # ------------------------------------------------ several volumes
    def _problems(self, problems):
        arr = (N.CsProblem * len(problems))()
        for i, p in enumerate(problems):
            arr[i] = p.cstruct()
        return arr

    def multi_step(self, problems, stream=None):
        """One Algorithm 1 iteration for each Problem; one traversal launch
        for all of them (cs_multi_step)."""
        arr = self._problems(problems)
        self._check("cs_multi_step", self.lib.cs_multi_step(self.h, arr, len(problems),
                                                            _stream(stream)))

    def multi_step_graph(self, problems) -> "Graph":
        arr = self._problems(problems)
        g = ctypes.c_void_p()
        self._check("cs_multi_step_graph",
                    self.lib.cs_multi_step_graph(self.h, arr, len(problems), ctypes.byref(g)))
        return Graph(self, g, problems)

    def set_slabs(self, slabs: int):
        """z-slabs per vector traversal (0: chosen from the grid's footprint)."""
        self._check("cs_set_slabs", self.lib.cs_set_slabs(self.h, int(slabs)))

    def set_host_mode(self, mode: str):
        """How precond_sgd_step_host moves a batch: "staged" (default) or
        "direct" (the traversal reads the images from device-mapped pinned
        memory; staged copies for other buffers)."""
        m = {"staged": N.CS_HOST_STAGED, "direct": N.CS_HOST_DIRECT}[mode]
        self._check("cs_set_host_mode", self.lib.cs_set_host_mode(self.h, m))

    def set_launch_shape(self, block_threads: int, blocks_per_sm: int):
        self._check("cs_set_launch_shape",
                    self.lib.cs_set_launch_shape(self.h, block_threads, blocks_per_sm))

    def autotune(self, problems):
        """(threads per block, blocks per SM) picked for these problems."""
        arr = self._problems(problems)
        bt, bps = ctypes.c_int(), ctypes.c_int()
        self._check("cs_autotune", self.lib.cs_autotune(self.h, arr, len(problems),
                                                        ctypes.byref(bt), ctypes.byref(bps)))
        return bt.value, bps.value

    # ------------------------------------------- learned preconditioner
    def mlp_forward(self, M, params, coverage, ctf2w, out=None, exp=False, offset=0.0,
                    tensor_cores=True, stream=None):
        if out is None:
            out = torch.empty((M, M, M), dtype=torch.float32, device=params.device)
        self._check("cs_mlp_forward", self.lib.cs_mlp_forward(
            self.h, M, _ptr(params, torch.float32, "params"),
            _ptr(coverage, torch.float32, "coverage"), _ptr(ctf2w, torch.float32, "ctf2w"),
            _ptr(out, torch.float32, "out"), int(exp), float(offset), int(tensor_cores),
            _stream(stream)))
        return out

    def mlp_target(self, M, estimates, floor_rel=1e-3, out=None, stream=None):
        """log of the mean of Hutchinson estimates [n_est][M][M][M], floored
        at floor_rel x the mean of the positive means (cs_mlp_target)."""
        if out is None:
            out = torch.empty((M, M, M), dtype=torch.float32, device=estimates.device)
        self._check("cs_mlp_target", self.lib.cs_mlp_target(
            self.h, M, int(estimates.shape[0]), _ptr(estimates, torch.float32, "estimates"),
            float(floor_rel), _ptr(out, torch.float32, "target"), _stream(stream)))
        return out

    def mlp_grad(self, M, r_ball, params, coverage, ctf2w, target, grad, sse,
                 tensor_cores=True, stream=None):
        self._check("cs_mlp_grad", self.lib.cs_mlp_grad(
            self.h, M, int(r_ball), _ptr(params, torch.float32, "params"),
            _ptr(coverage, torch.float32, "coverage"), _ptr(ctf2w, torch.float32, "ctf2w"),
            _ptr(target, torch.float32, "target"), _ptr(grad, torch.float32, "grad"),
            _ptr(sse, torch.float64, "sse"), int(tensor_cores), _stream(stream)))

    def mlp_adam_step(self, params, m, v, grad, step, lr=1e-2, beta1=0.9, beta2=0.999,
                      eps=1e-8, grad_scale=1.0, stream=None):
        self._check("cs_mlp_adam_step", self.lib.cs_mlp_adam_step(
            self.h, _ptr(params, torch.float32, "params"), _ptr(m, torch.float32, "m"),
            _ptr(v, torch.float32, "v"), _ptr(grad, torch.float32, "grad"), float(grad_scale),
            int(step), float(lr), float(beta1), float(beta2), float(eps), _stream(stream)))

    def check_device_status(self):
        self._check("cs_check_device_status", self.lib.cs_check_device_status(self.h))

    def selftest_wait_timeout(self, spins=1000, stream=None):
        """A bounded device-side wait that runs out: the next
        check_device_status raises with CS_ERR_TIMEOUT."""
        self._check("cs_selftest_wait_timeout",
                    self.lib.cs_selftest_wait_timeout(self.h, int(spins), _stream(stream)))

    def phase_shift(self, images, shifts, sign=-1, stream=None):
        """In place: images[i] *= T_i (sign +1) or conj(T_i) (sign -1)."""
        B, M = images.shape[0], images.shape[1]
        self._check("cs_phase_shift", self.lib.cs_phase_shift(
            self.h, M, _ptr(images, torch.complex64, "images"),
            _ptr(shifts, torch.float32, "shifts"), B, int(sign), _stream(stream)))
        return images

    def fsc(self, u, v, n_shells=None, stream=None):
        """Fourier shell correlation per shell; returns (fsc, sums) as device
        double tensors [n_shells] and [n_shells][3]."""
        M = u.shape[0]
        if n_shells is None:
            n_shells = M // 2
        sums = torch.empty((n_shells, 3), dtype=torch.float64, device=u.device)
        f = torch.empty(n_shells, dtype=torch.float64, device=u.device)
        self._check("cs_fsc", self.lib.cs_fsc(
            self.h, M, _ptr(u, torch.complex64, "u"), _ptr(v, torch.complex64, "v"),
            int(n_shells), _ptr(sums, torch.float64, "sums"), _ptr(f, torch.float64, "fsc"),
            _stream(stream)))
        return f, sums

    def shell_minmax(self, x, n_shells=None, stream=None):
        """Per-shell (min, max, count) of a real field [M][M][M]."""
        M = x.shape[0]
        if n_shells is None:
            n_shells = M // 2
        lo = torch.empty(n_shells, dtype=torch.float32, device=x.device)
        hi = torch.empty(n_shells, dtype=torch.float32, device=x.device)
        cnt = torch.empty(n_shells, dtype=torch.int32, device=x.device)
        self._check("cs_shell_minmax", self.lib.cs_shell_minmax(
            self.h, M, _ptr(x, torch.float32, "x"), int(n_shells),
            _ptr(lo, torch.float32, "min_out"), _ptr(hi, torch.float32, "max_out"),
            _ptr(cnt, torch.int32, "count_out"), _stream(stream)))
        return lo, hi, cnt

    def rel_err(self, geom: Geometry, v, v_ref, out=None, stream=None):
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=v.device)
        self._check("cs_rel_err", self.lib.cs_rel_err(
            self.h, geom.c, _ptr(v, torch.complex64, "v"), _ptr(v_ref, torch.complex64, "v_ref"),
            _ptr(out, torch.float64, "out"), _stream(stream)))
        return out


def disc_pixels(M: int, r_max: int) -> int:
    """Pixels of an M x M image inside the disc of radius r_max."""
    n = int(N.load().cs_disc_pixels(M, r_max))
    if n < 0:
        raise ValueError(f"M={M}, r_max={r_max} out of range")
    return n


def pack_disc(images: torch.Tensor, r_max: int) -> torch.Tensor:
    """images [B][M][M] -> their disc pixels [B][n_px] in the packed order of
    cs_precond_sgd_step_host_disc (row-major: ky ascending, then kx); a copy
    (data movement only)."""
    M = images.shape[-1]
    k = torch.arange(M) - M // 2
    mask = (k[:, None] ** 2 + k[None, :] ** 2) <= r_max * r_max
    return images[:, mask.to(images.device)].contiguous()


MODES = {"plain": N.CS_PLAIN, "hutchinson": N.CS_HUTCHINSON, "fixed": N.CS_FIXED}


class SGDState:
    """Algorithm 1 state on the device: v, D (init I), D_avg (init 0) and the
    scalar block (eta, k, alpha, loss, G, Q, halvings, status)."""

    def __init__(self, v0: torch.Tensor, mode="hutchinson", alpha=0.0, eta0=1.0, beta=0.9,
                 armijo_c=0.5, n_probes=1, seed=0, max_halvings=64, D=None):
        M = v0.shape[0]
        dev = v0.device
        self.v = v0.clone().contiguous()
        self.mode = mode
        self.D = (D.clone().contiguous() if D is not None
                  else torch.ones((M, M, M), dtype=torch.float32, device=dev))
        self.D_avg = torch.zeros((M, M, M), dtype=torch.float32, device=dev)
        self.scalars = torch.zeros(N.CS_NSCALARS, dtype=torch.float64, device=dev)
        self.scalars[N.CS_S_ETA] = eta0
        if torch.is_tensor(alpha):
            self.scalars[N.CS_S_ALPHA] = alpha.to(dev, torch.float64)
        else:
            self.scalars[N.CS_S_ALPHA] = float(alpha)
        self.n_probes, self.seed, self.beta = n_probes, seed, beta
        self.armijo_c = armijo_c
        self.max_halvings = max_halvings
        self._cs = None

    def cstruct(self) -> N.CsSgdState:
        s = N.CsSgdState()
        s.v = self.v.data_ptr()
        s.D = self.D.data_ptr()
        s.D_avg = self.D_avg.data_ptr()
        s.scalars = self.scalars.data_ptr()
        s.mode = MODES[self.mode]
        s.n_probes = self.n_probes
        s.seed = self.seed
        s.beta = self.beta
        s.c = self.armijo_c
        s.max_halvings = self.max_halvings
        self._cs = s
        return s

    # ------------------------------------------------------ checkpointing
    def state_dict(self) -> dict:
        """Everything Algorithm 1 carries between iterations: v, D, D_avg,
        the scalar block (eta, iteration count k, alpha, ...) and the
        hyper-parameters.  Probes are counter-based (iteration k uses probe
        block k + 1), so restoring this resumes the same trajectory."""
        return {"v": self.v.detach().cpu(), "D": self.D.detach().cpu(),
                "D_avg": self.D_avg.detach().cpu(), "scalars": self.scalars.detach().cpu(),
                "mode": self.mode, "n_probes": self.n_probes, "seed": self.seed,
                "beta": self.beta, "armijo_c": self.armijo_c, "max_halvings": self.max_halvings}

    @classmethod
    def from_state_dict(cls, sd: dict, device=None) -> "SGDState":
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        st = cls(sd["v"].to(dev), mode=sd["mode"], n_probes=sd["n_probes"], seed=sd["seed"],
                 beta=sd["beta"], armijo_c=sd["armijo_c"], max_halvings=sd["max_halvings"],
                 D=sd["D"].to(dev))
        st.D_avg.copy_(sd["D_avg"].to(dev))
        st.scalars.copy_(sd["scalars"].to(dev))
        return st

    def save(self, path: str):
        torch.save(self.state_dict(), path)

    @classmethod
    def load(cls, path: str, device=None) -> "SGDState":
        return cls.from_state_dict(torch.load(path, map_location="cpu"), device)


class Problem:
    """One refinement problem of a multi-volume step: geometry, SGD state and
    all of its images (n_batches batches of B) in device memory."""

    def __init__(self, geom: Geometry, state: SGDState, images, quat, defocus, B: int,
                 lam: float, scale: float):
        n_img = images.shape[0]
        if n_img % B:
            raise ValueError("the image count must be a multiple of B")
        for t, name in ((images, "images"), (quat, "quat")):
            _ptr(t, None, name)
        self.geom, self.state = geom, state
        self.images, self.quat, self.defocus = images, quat, defocus
        self.B, self.n_batches, self.lam, self.scale = B, n_img // B, lam, scale

    def cstruct(self) -> N.CsProblem:
        c = N.CsProblem()
        c.geom = self.geom._c
        c.state = self.state.cstruct()
        c.images = self.images.data_ptr()
        c.quat = self.quat.data_ptr()
        c.defocus = self.defocus.data_ptr() if self.defocus is not None else None
        c.B, c.n_batches = self.B, self.n_batches
        c.lam, c.scale = self.lam, self.scale
        return c


class Graph:
    """A captured multi-volume step; launch() replays one step."""

    def __init__(self, handle: Handle, g, problems):
        self.handle, self.g, self.problems = handle, g, problems

    def launch(self, stream=None):
        self.handle._check("cs_graph_launch",
                           self.handle.lib.cs_graph_launch(self.g, _stream(stream)))

    def close(self):
        if getattr(self, "g", None):
            self.handle.lib.cs_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
