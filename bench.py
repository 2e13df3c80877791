#!/usr/bin/env python
"""Throughput of the known-pose, preconditioned-SGD hot path on GB300.

A step is one iteration of Algorithm 1 (Toader, Brubaker & Lederman,
arXiv 2311.16100) on one mini-batch held in HBM: pose conversion, Hutchinson's
diagonal estimate (Eq. hutch, 32 Rademacher probes), the preconditioner update
and threshold (Eqs. diag est rule, thresh), the fused loss + gradient
(Eq. optim cp), the closed-form stochastic Armijo step (Eq. stochastic armijo)
and the update.  The default workload is a 128^3 complex64 Fourier volume of
1000 Gaussian blobs, 49152 synthetic 128x128 images (trilinear interpolation,
CTF 300 kV / Cs 2.7 mm / A 0.1 / 1.5 A, defocus U[1,3] um, SNR 0.05),
batch 1024; the metric is images per second through that step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
Under torchrun (N > 1) every rank runs an independent replica on its own
images (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grad images/s at N=128"
CONFIGS = {
    # name: grid side, images in HBM, batch, interpolation, probes, defocus (um), SNR, blobs
    "m128": dict(M=128, n_img=50000, B=1024, interp="trilinear", K=32, df=(1.0, 3.0),
                 snr=0.05, blobs=1000, seed=3000),
    "m64": dict(M=64, n_img=20000, B=256, interp="trilinear", K=32, df=(1.0, 3.0),
                snr=0.05, blobs=200, seed=2000),
    "m32": dict(M=32, n_img=1000, B=100, interp="nearest", K=16, df=None, snr=0.1,
                blobs=20, seed=1000),
    "m256": dict(M=256, n_img=100000, B=1024, interp="trilinear", K=32, df=(1.0, 3.0),
                 snr=0.05, blobs=5000, seed=5000),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    p.add_argument("--config", choices=sorted(CONFIGS), default="m128")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-metric2", action="store_true",
                   help="skip the time-to-relative-error runs (plain vs preconditioned)")
    p.add_argument("--mlp-only", action="store_true",
                   help="only time the learned-preconditioner network kernels at 128^3")
    p.add_argument("--no-learned", action="store_true",
                   help="skip the learned-preconditioner leg")
    p.add_argument("--no-graph", action="store_true",
                   help="skip the single-problem CUDA-graph replay figure")
    p.add_argument("--no-loss-grad", action="store_true",
                   help="skip the cs_loss_grad-only throughput")
    p.add_argument("--no-multi", action="store_true",
                   help="skip the multi-volume graph-replay throughput")
    p.add_argument("--cpu-sample", type=int, default=128,
                   help="images in the oracle's timed sample")
    p.add_argument("--algo", choices=["auto", "vector", "tiled", "pixel"], default="auto",
                   help="scatter algorithm of the adjoint-type passes")
    p.add_argument("--images", type=int, default=0,
                   help="override the number of images held in HBM (profiling runs)")
    p.add_argument("--config-file", default=None,
                   help="JSON object whose keys override the named workload's fields "
                        "(M, n_img, B, interp, K, df, snr, blobs, seed)")
    return p.parse_args()


def workload_config(args):
    """The named workload, with the fields of --config-file (a JSON object)
    and --images applied on top."""
    cfg = dict(CONFIGS[args.config])
    if getattr(args, "config_file", None):
        with open(args.config_file) as f:
            extra = json.load(f)
        unknown = set(extra) - set(cfg)
        if unknown:
            raise SystemExit(f"--config-file: unknown workload fields {sorted(unknown)}")
        if "df" in extra and extra["df"] is not None:
            extra["df"] = tuple(extra["df"])
        cfg.update(extra)
    if args.images:
        cfg["n_img"] = max(cfg["B"], args.images)
    return cfg


# ------------------------------------------------------------------ helpers
def n_disc_pixels(M, r):
    k = range(-(M // 2), M // 2)
    return sum(1 for y in k for x in k if x * x + y * y <= r * r)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# sources that define the kernel of each timed phase (for the validity of
# recorded ncu counters)
KERNEL_SOURCES = {
    "loss_grad": ["fused.cu", "fused.h", "fused_ws.h", "device.cuh"],
    "curvature": ["fused.cu", "fused.h", "fused_ws.h", "device.cuh"],
}


def kernel_source_hash(kernel="loss_grad"):
    """Hash of the code of the kernel's sources: line comments, trailing
    blanks and empty lines are left out, so that a comment edit keeps the
    recorded counters valid and any code edit voids them."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_16100_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or sorted(
        f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h")))
    for f in files:
        for line in open(os.path.join(csrc, f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(config, kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = rec.get(f"{kernel}:{config}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """SM clock and clock-event (throttle) reasons of the benchmark's GPU,
    polled through NVML every ~2 ms in a background thread (read-only NVML
    queries; no setting is changed)."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import ctypes
        self.ok = False
        self.samples = []
        self.reasons = 0
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            bus = None
            try:
                import torch
                p = torch.cuda.get_device_properties(torch_device)
                bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
            except Exception:
                bus = None
            rc = 1
            if bus:
                rc = self.nvml.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.dev))
            if rc != 0:
                rc = self.nvml.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(self.dev))
            if rc != 0:
                return
            mx = ctypes.c_uint()
            self.nvml.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx))
            self.max_mhz = mx.value
            self.ok = True
        except OSError:
            pass

    def _poll(self):
        import ctypes
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        get_r = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag:
            if self.nvml.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if get_r(self.dev, ctypes.byref(rs)) == 0:
                self.reasons |= rs.value
            time.sleep(0.002)

    def start(self):
        if not self.ok:
            return
        self.stop_flag = False
        self.t = threading.Thread(target=self._poll, daemon=True)
        self.t.start()

    def stop(self):
        if not self.ok:
            return None
        self.stop_flag = True
        self.t.join(timeout=2)
        if not self.samples:
            return None
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in sorted(self.REASONS.items()) if self.reasons & b],
                "samples": len(self.samples), "source": "nvml"}


# ------------------------------------------------------- replicas (N > 1)
def replica_seed(cfg, rank):
    """Each rank runs an independent replica on its own seeded dataset."""
    return cfg["seed"] + 100 * rank


def max_over_ranks(values, world, device="cuda"):
    """Element-wise maximum over ranks (the slowest replica sets the time)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_value(world, batch, steps, ms):
    """Whole-job throughput: images processed by all ranks / the max time."""
    return world * batch * steps / (ms / 1e3)


# ------------------------------------------------------------------ GPU arm
def batches(n_img, B):
    """(start, size) of each mini-batch over a dataset of n_img images taken in
    order: full batches of B and, when B does not divide n_img, a short last
    one (its step uses the scale n_img / size, the batch reading of Eq. optim
    cp)."""
    return [(s, min(B, n_img - s)) for s in range(0, n_img, B)]


def build_workload(cfg, rank, h, torch, ops, synth):
    M, B = cfg["M"], cfg["B"]
    n_img = cfg["n_img"]
    bl = batches(n_img, B)
    dev = torch.device("cuda", torch.cuda.current_device())
    ctf = ops.CTF() if cfg["df"] else None
    geom = ops.Geometry(M, M // 2 - 1, cfg["interp"], ctf)
    seed = replica_seed(cfg, rank)
    v_true = torch.from_numpy(synth.blob_volume(M, cfg["blobs"], seed=seed)).to(dev)
    quat = torch.from_numpy(synth.shoemake_quaternions(n_img, seed + 1).astype("float32")).to(dev)
    if cfg["df"]:
        df = torch.from_numpy(synth.defocus_angstrom(n_img, seed + 2, *cfg["df"])
                              .astype("float32")).to(dev)
    else:
        df = torch.zeros(n_img, dtype=torch.float32, device=dev)
    images = torch.empty((n_img, M, M), dtype=torch.complex64, device=dev)
    rot = torch.empty((B, 3, 3), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 3)
    disc = torch.from_numpy(synth.ball_mask(M, M // 2 - 1)[M // 2]).to(dev)
    sig2 = None
    for start, size in bl:
        sl = slice(start, start + size)
        h.quat_to_rot(quat[sl], rot[:size])
        clean = h.slice_project(geom, v_true, rot[:size], df[sl] if ctf else None,
                                out=images[sl])
        if sig2 is None:
            sig2 = float((clean.abs() ** 2)[:, disc].mean()) / cfg["snr"]
        noise = torch.randn((size, M, M), dtype=torch.complex64, device=dev, generator=gen)
        images[sl] += noise * (sig2 ** 0.5) * disc.to(torch.complex64)
    torch.cuda.synchronize()
    return dict(geom=geom, v_true=v_true, quat=quat, df=df, images=images, rot=rot, nb=len(bl),
                batches=bl, n_img=n_img, sigma2=sig2, ctf=ctf)


def run_gpu(args, cfg, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2311_16100_gb300 import ops, synth
    from paper_2311_16100_gb300 import native as N

    h = ops.Handle(torch.cuda.current_device())
    h.set_algo(args.algo)
    W = build_workload(cfg, rank, h, torch, ops, synth)
    M, B, nb, bl = cfg["M"], cfg["B"], W["nb"], W["batches"]
    geom, images, quat, df, rot = W["geom"], W["images"], W["quat"], W["df"], W["rot"]
    lam = W["sigma2"]                       # lambda = sigma^2 / tau^2 with tau^2 = 1
    scale = W["n_img"] / B
    alpha = h.threshold_alpha(geom, df if W["ctf"] else None, W["n_img"], lam)
    v0 = torch.from_numpy(synth.initial_volume(M, M // 2 - 1, 1.0, cfg["seed"] + 7)).cuda()
    st = ops.SGDState(v0, mode="hutchinson", alpha=alpha, eta0=1.0, beta=0.9, armijo_c=0.5,
                      n_probes=cfg["K"], seed=cfg["seed"] + 11)
    h.reserve(M, B)
    dfs = (lambda sl: df[sl]) if W["ctf"] else (lambda sl: None)

    def step(s):
        start, size = bl[s % nb]
        sl = slice(start, start + size)
        h.quat_to_rot(quat[sl], rot[:size])
        h.precond_sgd_step(geom, st, images[sl], rot[:size], dfs(sl), lam, W["n_img"] / size)
        return size

    stream = torch.cuda.current_stream()
    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    l0 = ops.kernel_launches()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    timed_images = 0
    for s in range(args.warmup, args.warmup + args.steps):
        timed_images += step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = ops.kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    # phase breakdown from a second run of as many steps with the library's
    # event profiler on (kept out of the timed loop above)
    h.profile_enable(True, args.steps)
    prof_images = 0
    for s in range(args.warmup + args.steps, args.warmup + 2 * args.steps):
        prof_images += step(s)
    torch.cuda.synchronize()
    phases = h.profile_read()
    h.profile_enable(False)
    sc = st.scalars.cpu().tolist()
    ms = max_over_ranks([ms], world)[0]

    # --- end to end through the public API with host buffers: every step
    # copies its batch from pinned host memory (cs_precond_sgd_step_host,
    # double-buffered: the copy of batch n+1 overlaps step n) and reads the
    # batch loss back into pinned host memory
    e2e = None
    if not args.no_e2e:
        nh = min(4, nb)
        pin_img = [images[i * B:(i + 1) * B].cpu().pin_memory() for i in range(nh)]
        # the same batches as their disc pixels only (the layout of
        # cs_precond_sgd_step_host_disc)
        pin_disc = [ops.pack_disc(images[i * B:(i + 1) * B], M // 2 - 1).cpu().pin_memory()
                    for i in range(nh)]
        pin_q = [quat[i * B:(i + 1) * B].cpu().pin_memory() for i in range(nh)]
        pin_df = [df[i * B:(i + 1) * B].cpu().pin_memory() for i in range(nh)]
        out_loss = torch.zeros(max(args.steps, args.warmup), dtype=torch.float64).pin_memory()

        def e2e_step(s, i, disc=False):
            j = s % nh
            if disc:
                h.precond_sgd_step_host_disc(geom, st, pin_disc[j], pin_q[j],
                                             pin_df[j] if W["ctf"] else None, lam, scale,
                                             loss_host=out_loss[i])
            else:
                h.precond_sgd_step_host(geom, st, pin_img[j], pin_q[j],
                                        pin_df[j] if W["ctf"] else None, lam, scale,
                                        loss_host=out_loss[i])

        def e2e_run(mode):
            disc = mode == "disc"
            h.set_host_mode("staged" if disc else mode)
            for s in range(args.warmup):
                e2e_step(s, s, disc)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0 = time.perf_counter()
            a0.record(stream)
            for i in range(args.steps):
                e2e_step(i, i, disc)
            a1.record(stream)
            torch.cuda.synchronize()
            wall_ = (time.perf_counter() - w0) * 1e3
            ems_ = a0.elapsed_time(a1)
            ems_, wall_ = max_over_ranks([ems_, wall_], world)
            assert bool(torch.isfinite(out_loss[: args.steps]).all()) and float(out_loss[0]) != 0.0
            return ems_, wall_

        # the images as their disc pixels (staged), the full images (staged
        # copies), then the direct reads of the full images from the pinned
        # buffers over the host link
        ems, wall = e2e_run("disc")
        ems_full, _ = e2e_run("staged")
        ems_dir, _ = e2e_run("direct")
        h.set_host_mode("staged")
        # the host-to-device rate alone: the same batches copied back to back
        # with nothing else running (the rate the end-to-end steps depend on)
        dev_img = torch.empty_like(images[:B])
        cs_ = torch.cuda.Stream()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(cs_):
            dev_img.copy_(pin_img[0], non_blocking=True)
            c0.record(cs_)
            for i in range(args.steps):
                dev_img.copy_(pin_img[i % nh], non_blocking=True)
            c1.record(cs_)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / args.steps
        del dev_img
        n_px_disc = ops.disc_pixels(M, M // 2 - 1)
        e2e = {"value": job_value(world, B, args.steps, ems), "unit": "images/s",
               "h2d_bytes_per_step": B * n_px_disc * 8 + B * 16 + B * 4,
               "d2h_bytes_per_step": 8,
               "host_wall_value": round(job_value(world, B, args.steps, wall), 1),
               "full_images_value": job_value(world, B, args.steps, ems_full),
               "full_images_h2d_bytes_per_step": B * M * M * 8 + B * 16 + B * 4,
               "h2d_copy_only": {"GB_per_s": round(B * M * M * 8 / (cms / 1e3) / 1e9, 1),
                                 "images_per_s_at_that_rate": round(world * B / (cms / 1e3), 1)},
               "direct_value": job_value(world, B, args.steps, ems_dir),
               "api": "cs_precond_sgd_step_host_disc (images as their disc pixels, "
                      "double-buffered staging copies on a copy stream); full_images_value: "
                      "cs_precond_sgd_step_host with whole images; direct_value: the "
                      "traversal reading the disc pixels from the pinned full images instead"}

    # --- roofline of the dominant phase
    n_px = n_disc_pixels(M, M // 2 - 1)
    hutch = cfg["K"] > 0
    Bp = prof_images / args.steps           # images per launch, averaged over the profiled steps
    alg_bytes = {   # algorithmic DRAM bytes of one launch of each phase
        # fused traversal: images + poses read once, volume read, gradient
        # (and Hutchinson diagonal) written once
        "loss_grad": round(Bp * (8 * n_px + 36 + 4)) + M ** 3 * (8 + 8 + (4 if hutch else 0)),
        "precond": M ** 3 * (8 + 16),
        "direction": M ** 3 * (8 + 8 + 4 * 5 + 16),
        "curvature": round(Bp * (36 + 4)) + 16 * M ** 3,
        "update": M ** 3 * (16 + 8 + 8),
    }
    # 16-byte reductions per pixel of the trilinear fused pass: 4 for the
    # complex gradient, 2 for the Hutchinson diagonal
    reds = {"loss_grad": round(Bp * n_px * (4 + (2 if hutch else 0)))}
    per = {k: v[0] / max(v[1], 1) for k, v in phases.items()}
    dom = max(per, key=per.get)
    peaks, peak_src = measured_peaks()
    ach = alg_bytes[dom] / (per[dom] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1),
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
            "peak_source": peak_src,
            "traffic": recorded_traffic(args.config, dom),
            "algorithmic_bytes": alg_bytes[dom], "ms_per_launch": round(per[dom], 4)}
    red_roof = None
    if dom in reds and cfg["interp"] == "trilinear":
        red_peak = h.measure_reduction_rate()
        red_ach = reds[dom] / (per[dom] / 1e3) / 1e9
        red_roof = {"bound": "l2_reductions", "kernel": dom, "achieved": round(red_ach, 1),
                    "peak": round(red_peak, 1), "unit": "G reductions/s",
                    "frac": round(red_ach / red_peak, 4),
                    "peak_source": "cs_measure_reduction_rate, live",
                    "reductions_per_launch": reds[dom]}
    # the same steps replayed as a CUDA graph (batch k mod n_batches chosen
    # on the device), launch shape from the autotuner
    graph = None
    if not args.no_graph and world == 1:
        st_g = ops.SGDState(v0, mode="hutchinson", alpha=alpha, eta0=1.0, beta=0.9,
                            armijo_c=0.5, n_probes=cfg["K"], seed=cfg["seed"] + 11)
        n_full = W["n_img"] // B * B        # the device-side batch cursor takes full batches
        prob = ops.Problem(geom, st_g, images[:n_full], quat[:n_full],
                           df[:n_full] if W["ctf"] else None, B, lam, W["n_img"] / B)
        hg = ops.Handle(torch.cuda.current_device())
        bt, bps = hg.autotune([prob])
        gr = hg.multi_step_graph([prob])
        for _ in range(args.warmup):
            gr.launch(stream)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            gr.launch(stream)
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / args.steps
        graph = {"ms_per_step": round(gms, 4), "images_per_s": round(B / (gms / 1e3), 1),
                 "batches": f"{n_full // B} full batches of {B}",
                 "launch_shape": {"block_threads": bt, "blocks_per_sm": bps},
                 "api": "cs_multi_step_graph with one problem, cs_graph_launch"}
        gr.close()
        hg.close()
    # cs_loss_grad alone (loss and gradient, no Hutchinson, no step): median
    # over 20 passes of the per-batch time, every batch of the image set
    lg = None
    if not args.no_loss_grad:
        g_buf = torch.empty_like(st.v)
        l_buf = torch.empty((), dtype=torch.float64, device="cuda")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(20)]
        for _ in range(3):
            h.loss_grad(geom, st.v, images[:B], rot, dfs(slice(0, B)), lam, scale, grad=g_buf,
                        loss=l_buf)
        per_pass = []
        for i in range(20):
            ev[i][0].record(stream)
            for start, size in bl:
                sl = slice(start, start + size)
                h.quat_to_rot(quat[sl], rot[:size])
                h.loss_grad(geom, st.v, images[sl], rot[:size], dfs(sl), lam,
                            W["n_img"] / size, grad=g_buf, loss=l_buf)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        per_pass = sorted(a.elapsed_time(b_) for a, b_ in ev)
        med = per_pass[len(per_pass) // 2]
        ips = W["n_img"] / (med / 1e3)
        npx = n_disc_pixels(M, M // 2 - 1)
        # byte rates the images/s stand for: per image, its disc pixels and
        # pose from HBM; in L2 the trilinear gathers (8 corners x 8 bytes)
        # and the adjoint's additions (8 corners x 8 bytes) per pixel
        lg = {"metric": "cs_loss_grad images/s (loss + gradient only)",
              "value": round(ips, 1), "unit": "images/s",
              "ms_per_pass_median": round(med, 4), "passes": 20,
              "pass": f"{W['n_img']} images in {nb} batches of up to {B} (every image once), "
                      "poses converted per batch",
              "hbm_GB_per_s_equivalent": round(ips * (8 * npx + 20) / 1e9, 1),
              "l2_GB_per_s_equivalent": round(ips * (64 + 64) * npx / 1e9, 1)}
    return dict(ms=ms, timed_images=timed_images, launches=launches, phases={k: round(v, 4) for k, v in per.items()},
                roofline=roof, red_roofline=red_roof, e2e=e2e, clocks=clk, scalars=sc, n_img=W["n_img"],
                loss_grad_only=lg, graph=graph)


# ------------------------------------------- time to relative error (metric 2)
TTE_CONFIGS = {
    # Fourier volume, images, batch, epochs as in the refinement workloads
    "m32_nearest": dict(M=32, n_img=1000, B=100, epochs=5, interp="nearest", K=16, df=None,
                        snr=0.1, blobs=20, seed=1000),
    "m64_trilinear_ctf": dict(M=64, n_img=20480, B=256, epochs=10, interp="trilinear", K=32,
                              df=(1.0, 3.0), snr=0.05, blobs=200, seed=2000),
    # the same problems with little image noise (SNR 10): the mini-batch
    # noise floor drops and the conditioning of H decides the speed
    "m32_nearest_snr10": dict(M=32, n_img=1000, B=100, epochs=5, interp="nearest", K=16,
                              df=None, snr=10.0, blobs=20, seed=1000),
    "m64_trilinear_ctf_snr10_b1024": dict(M=64, n_img=20480, B=1024, epochs=20,
                                          interp="trilinear", K=32, df=(1.0, 3.0), snr=10.0,
                                          blobs=200, seed=2000),
}
THRESHOLDS = [0.5, 0.3, 0.2, 0.15, 0.1, 0.05, 0.02, 0.01]
# the learned preconditioner's features come from the first 1/8 of a
# dataset's poses (scaled to the whole dataset), in training and in use
FEATURE_SUBSAMPLE = 8


def ground_truth(h, torch, synth, W, cfg, lam):
    """v* solving H v = b over the whole dataset: closed form under nearest
    interpolation, conjugate gradients with the library's gradient otherwise."""
    M = cfg["M"]
    r = M // 2 - 1
    geom, images, quat, df = W["geom"], W["images"], W["quat"], W["df"]
    dfa = df if W["ctf"] else None
    rot_all = h.quat_to_rot(quat)
    b = h.backproject_adjoint(geom, images, rot_all, dfa, 1.0)
    ball = torch.from_numpy(synth.ball_mask(M, r)).cuda()
    if cfg["interp"] == "nearest":
        d, _, _ = h.exact_diag(geom, rot_all, dfa, lam, 1.0)
        return torch.where(ball, b / d, torch.zeros_like(b)), rot_all
    zeros = torch.zeros_like(images)
    x = torch.zeros_like(b)
    rr = b.clone()
    pp = rr.clone()
    rs = float(torch.sum(torch.abs(rr) ** 2))
    bn = rs ** 0.5
    for _ in range(500):
        _, Hp = h.loss_grad(geom, pp, zeros, rot_all, dfa, lam, 1.0)
        a = rs / float(torch.sum((torch.conj(pp) * Hp).real))
        x += a * pp
        rr -= a * Hp
        rs_new = float(torch.sum(torch.abs(rr) ** 2))
        if rs_new ** 0.5 <= 1e-6 * bn:
            break
        pp = rr + (rs_new / rs) * pp
        rs = rs_new
    del zeros
    return torch.where(ball, x, torch.zeros_like(x)), rot_all


def sgd_arms(h, torch, ops, synth, W, cfg, vstar, lam, arms, epochs):
    """Algorithm 1 from the same start for each arm ({name: (mode, D)}):
    device time of the steps to reach each relative error (evaluated after
    every step outside the timing), and the Fourier shell correlation with
    v* after every epoch at a low, a middle and a high shell."""
    M, B = cfg["M"], cfg["B"]
    r = M // 2 - 1
    geom, images, quat, df, n_img = W["geom"], W["images"], W["quat"], W["df"], W["n_img"]
    alpha = h.threshold_alpha(geom, df if W["ctf"] else None, n_img, lam)
    v0 = torch.from_numpy(synth.initial_volume(M, r, 1.0, cfg["seed"] + 7)).cuda()
    out = {}
    for name, (mode, D) in arms.items():
        st = ops.SGDState(v0, mode=mode, alpha=alpha, eta0=1.0, beta=0.9, armijo_c=0.5,
                          n_probes=cfg["K"], seed=cfg["seed"] + 11, D=D)
        err = h.rel_err(geom, st.v, vstar)
        first = {t: None for t in THRESHOLDS}
        t_ms = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rot = torch.empty((B, 3, 3), dtype=torch.float32, device="cuda")
        shells = (M // 16, M // 4, M // 2 - 2)
        fsc_ep = {str(r_): [] for r_ in shells}
        for ep in range(epochs):
            perm = torch.from_numpy(synth.permutation(n_img, cfg["seed"] + 31 + ep)).cuda()
            im_p, q_p = images[perm].contiguous(), quat[perm].contiguous()
            df_p = df[perm].contiguous() if W["ctf"] else None
            torch.cuda.synchronize()
            for start, size in batches(n_img, B):
                sl = slice(start, start + size)
                e0.record()
                h.quat_to_rot(q_p[sl], rot[:size])
                h.precond_sgd_step(geom, st, im_p[sl], rot[:size],
                                   df_p[sl] if df_p is not None else None, lam, n_img / size)
                e1.record()
                h.rel_err(geom, st.v, vstar, out=err)
                torch.cuda.synchronize()
                t_ms += e0.elapsed_time(e1)
                e = float(err)
                for t in THRESHOLDS:
                    if first[t] is None and e <= t:
                        first[t] = round(t_ms, 3)
            del im_p, q_p, df_p
            f, _ = h.fsc(st.v, vstar, M // 2)          # Eq. fsc against v*, per epoch
            f = f.cpu().numpy()
            for r_ in shells:
                fsc_ep[str(r_)].append(round(float(f[r_]), 4))
        below = [r_ for r_ in range(1, M // 2) if f[r_] < 0.5]
        out[name] = {"ms_to_rel_err": {str(t): first[t] for t in THRESHOLDS},
                     "reached_1e-2": first[0.01] is not None,
                     "final_rel_err": round(float(err), 5), "total_ms": round(t_ms, 3),
                     "final_eta": float(st.scalars[0]),
                     "fsc_by_epoch_at_shell": fsc_ep,
                     "first_shell_fsc_below_0.5": below[0] if below else None}
    return out


def time_to_error(cfg, torch, ops, synth, h):
    """Wall (device) time of Algorithm 1 to reach relative volume errors,
    plain SGD vs Hutchinson-preconditioned, both with the Armijo rule."""
    W = build_workload(dict(cfg, n_img=cfg["n_img"]), 0, h, torch, ops, synth)
    lam = W["sigma2"]
    vstar, rot_all = ground_truth(h, torch, synth, W, cfg, lam)
    D_pre, pre = precomputed(h, torch, W, rot_all, cfg, lam)
    out = {"workload": f"{cfg['M']}^3, {W['n_img']} images, batch {cfg['B']}, "
                       f"{cfg['epochs']} epochs, {cfg['interp']}, "
                       f"{'CTF' if cfg['df'] else 'no CTF'}, {cfg['K']} probes", "lambda": lam,
           "precomputed_setup": pre}
    out.update(sgd_arms(h, torch, ops, synth, W, cfg, vstar, lam,
                        {"plain": ("plain", None), "precomputed": ("fixed", D_pre),
                         "hutchinson": ("hutchinson", None)},
                        cfg["epochs"]))
    return out


def precomputed(h, torch, W, rot_all, cfg, lam):
    """Section 4's precomputed preconditioner: Eq. diag est rule over
    ceil(1000/K) epochs of K-probe batch estimates (as many probe draws per
    image as the paper's 1000 single-probe epochs)."""
    epochs = -(-1000 // cfg["K"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    D = h.precompute_preconditioner(W["geom"], rot_all, W["df"] if W["ctf"] else None,
                                    B=cfg["B"], n_epochs=epochs, lam=lam, n_probes=cfg["K"],
                                    seed=cfg["seed"] + 13)
    e1.record()
    torch.cuda.synchronize()
    return D, {"epochs": epochs, "probes_per_batch": cfg["K"], "ms": round(e0.elapsed_time(e1), 3)}


def mlp_kernels(h, torch, M, r, params, cov, c2w, target):
    """Device time of the network's forward (inference over the M^3 grid) and
    gradient kernels, tensor-core and FP32 reference, and the forward's
    tensor roofline.  Algorithmic FLOPs per voxel: forward 2 (3*64 + 64*64 +
    64) = 8704; gradient adds the 64 x 64 backward product and the weight
    Gram product (2 * 2 * 64*64) and the small layers (2 * (3*64 + 64*3)),
    25,472 in all; both kernels process every voxel of the grid."""
    dev = params.device
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out_buf = torch.empty((M, M, M), device=dev)
    res = {}
    for tc in (True, False):
        for _ in range(3):
            h.mlp_forward(M, params, cov, c2w, out=out_buf, tensor_cores=tc)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            h.mlp_forward(M, params, cov, c2w, out=out_buf, tensor_cores=tc)
        e1.record()
        torch.cuda.synchronize()
        fwd = e0.elapsed_time(e1) / 10
        g = torch.zeros_like(params)
        sse = torch.zeros((), dtype=torch.float64, device=dev)
        for _ in range(3):
            h.mlp_grad(M, r, params, cov, c2w, target, g, sse, tc)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            h.mlp_grad(M, r, params, cov, c2w, target, g, sse, tc)
        e1.record()
        torch.cuda.synchronize()
        grd = e0.elapsed_time(e1) / 10
        res["tensor_cores" if tc else "fp32_reference"] = {"forward_ms": round(fwd, 4),
                                                           "gradient_ms": round(grd, 4)}
    h.check_device_status()
    nvox = M ** 3
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    fwd_flops = nvox * 2 * (3 * 64 + 64 * 64 + 64)
    grad_flops = nvox * 2 * (3 * 64 + 3 * 64 * 64 + 64 + 64 * 3)
    tcf = res["tensor_cores"]
    ach = fwd_flops / (tcf["forward_ms"] / 1e3) / 1e12
    ach_g = grad_flops / (tcf["gradient_ms"] / 1e3) / 1e12
    roof = {"bound": "tensor", "kernel": "k_mlp_forward_tc", "achieved": round(ach, 2),
            "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 5),
            "peak_source": src, "flops_per_launch": fwd_flops,
            "gradient": {"kernel": "k_mlp_grad_tc", "achieved": round(ach_g, 2),
                         "frac": round(ach_g / peak, 5), "flops_per_launch": grad_flops}}
    return res, roof


def mlp_only(args):
    """Only the network kernels at 128^3 on seeded features (random weights)."""
    import torch
    from paper_2311_16100_gb300 import ops
    from paper_2311_16100_gb300.learned import init_params
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    h = ops.Handle(0)
    M, r = 128, 63
    g = torch.Generator(device="cpu")
    g.manual_seed(4242)
    cov = (torch.rand((M, M, M), generator=g) * 400).to(dev)
    c2w = (torch.rand((M, M, M), generator=g) * 200).to(dev)
    target = torch.randn((M, M, M), generator=g).to(dev)
    params = torch.from_numpy(init_params(7)).to(dev)
    res, roof = mlp_kernels(h, torch, M, r, params, cov, c2w, target)
    print(json.dumps({"workload": "learned-preconditioner network, 128^3 voxels",
                      "kernels": res, "roofline": roof}), flush=True)
    h.close()


def learned_leg(args, torch, ops, synth):
    """The learned preconditioner: trained on Hutchinson estimates from 8
    seeded 128^3 pose sets (50k poses each, defocus U[0.5, 3.5] um), its
    kernels timed against the tensor roofline, its D compared with the exact
    diagonal, and SGD preconditioned by it raced against Algorithm 1 and
    plain SGD on the benchmark's dataset."""
    from paper_2311_16100_gb300.learned import (LearnedPreconditioner, Sample, dataset_features,
                                                hutchinson_target)
    h = ops.Handle(torch.cuda.current_device())
    M, r = 128, 63
    geom = ops.Geometry(M, r, "trilinear", ops.CTF())
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    samples = []
    for s_ in range(8):
        q = torch.from_numpy(synth.shoemake_quaternions(50000, 8000 + 10 * s_)
                             .astype("float32")).to(dev)
        rot = h.quat_to_rot(q)
        df = torch.from_numpy(synth.defocus_angstrom(50000, 8001 + 10 * s_, 0.5, 3.5)
                              .astype("float32")).to(dev)
        cov, c2w = dataset_features(h, geom, rot, df, subsample=FEATURE_SUBSAMPLE)
        samples.append(Sample(M, r, cov, c2w, hutchinson_target(h, geom, rot, df)))
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = LearnedPreconditioner(h, seed=1)
    t0 = time.perf_counter()
    hist = net.fit(samples, steps=300, lr=1e-2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    s0 = samples[0]
    res, mlp_roof = mlp_kernels(h, torch, M, r, net.params, s0.coverage, s0.ctf2w, s0.target)
    # the benchmark's dataset (and the same poses with little image noise):
    # D from the network (one pose-only feature pass and one inference) vs
    # the exact diagonal, then the SGD race
    out = None
    for snr in (CONFIGS["m128"]["snr"], 10.0):
        race = learned_race(h, torch, ops, synth, net, geom, samples, hist, t_data, t_train, res,
                            mlp_roof, snr)
        if out is None:
            out = race
        else:
            out["time_to_rel_err_snr10"] = race["time_to_rel_err"]
    # the network trained on 128^3 pose sets, applied to a 64^3 problem
    # (its features are normalised): SNR 10, batch 4096 (5 steps per epoch),
    # 120 epochs, long enough for the preconditioned arms to pass 1e-2
    cfg = dict(TTE_CONFIGS["m64_trilinear_ctf_snr10_b1024"], epochs=120, B=4096)
    W = build_workload(cfg, 0, h, torch, ops, synth)
    lam = W["sigma2"]
    vstar, rot_all = ground_truth(h, torch, synth, W, cfg, lam)
    # each fixed preconditioner's set-up on this dataset (device time)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    cov, c2w = dataset_features(h, W["geom"], rot_all, W["df"], subsample=FEATURE_SUBSAMPLE)
    D_learned = net.predict(64, cov, c2w, lam)
    e1.record()
    torch.cuda.synchronize()
    setup = {"learned": round(e0.elapsed_time(e1), 3)}
    e0.record()
    exact, _, _ = h.exact_diag(W["geom"], rot_all, W["df"], lam, 1.0)
    e1.record()
    torch.cuda.synchronize()
    setup["exact_diagonal_control"] = round(e0.elapsed_time(e1), 3)
    D_pre, pre = precomputed(h, torch, W, rot_all, cfg, lam)
    setup["precomputed"] = pre["ms"]
    arms = {"plain": ("plain", None), "precomputed": ("fixed", D_pre),
            "hutchinson": ("hutchinson", None), "learned": ("fixed", D_learned),
            "exact_diagonal_control": ("fixed", exact)}
    r64 = sgd_arms(h, torch, ops, synth, W, cfg, vstar, lam, arms, cfg["epochs"])
    r64["setup_ms"] = setup
    r64["workload"] = (f"64^3, {W['n_img']} images, batch 4096, 120 epochs, trilinear, CTF, "
                       "SNR 10, 32 probes; network trained on 128^3 pose sets")
    out["time_to_rel_err_64_snr10_b4096"] = r64
    del W
    h.close()
    return out


def learned_race(h, torch, ops, synth, net, geom, samples, hist, t_data, t_train, res, mlp_roof,
                 snr):
    from paper_2311_16100_gb300.learned import dataset_features
    M, r = 128, 63
    dev = torch.device("cuda", torch.cuda.current_device())
    cfg = dict(CONFIGS["m128"], epochs=10, snr=snr)
    W = build_workload(cfg, 0, h, torch, ops, synth)
    lam = W["sigma2"]
    vstar, rot_all = ground_truth(h, torch, synth, W, cfg, lam)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    cov, c2w = dataset_features(h, geom, rot_all, W["df"], subsample=FEATURE_SUBSAMPLE)
    D_learned = net.predict(M, cov, c2w, lam)
    e1.record()
    torch.cuda.synchronize()
    setup_learned = e0.elapsed_time(e1)
    e0.record()
    exact, _, _ = h.exact_diag(geom, rot_all, W["df"], lam, 1.0)
    e1.record()
    torch.cuda.synchronize()
    setup_exact = e0.elapsed_time(e1)
    ball = torch.from_numpy(synth.ball_mask(M, r)).to(dev)
    rel = lambda a, b: float(torch.linalg.vector_norm((a - b)[ball]) /
                             torch.linalg.vector_norm(b[ball]))
    per = len(samples) * samples[0].n_ball
    out = {"training": {"datasets": "8 x 50000 poses, 128^3, defocus U[0.5,3.5] um",
                        "targets": "log of Hutchinson estimates, 4 x 32 probes",
                        "features": f"from 1/{FEATURE_SUBSAMPLE} of each dataset's poses",
                        "adam_steps": len(hist), "mse_first": hist[0] / per,
                        "mse_last": hist[-1] / per,
                        "data_s": round(t_data, 3), "train_s": round(t_train, 3)},
           "kernels_128cubed": res, "roofline": mlp_roof,
           "D_rel_err_vs_exact": round(rel(D_learned, exact), 4),
           "setup_ms": {"learned": round(setup_learned, 3),
                        "exact_diagonal_control": round(setup_exact, 3)}}
    D_pre, pre = precomputed(h, torch, W, rot_all, cfg, lam)
    out["setup_ms"]["precomputed"] = pre["ms"]
    out["D_rel_err_vs_exact_precomputed"] = round(rel(D_pre, exact), 4)
    arms = {"plain": ("plain", None), "precomputed": ("fixed", D_pre),
            "hutchinson": ("hutchinson", None), "learned": ("fixed", D_learned),
            "exact_diagonal_control": ("fixed", exact)}
    out["time_to_rel_err"] = sgd_arms(h, torch, ops, synth, W, cfg, vstar, lam, arms,
                                      cfg["epochs"])
    out["time_to_rel_err"]["workload"] = (f"128^3, {W['n_img']} images, batch 1024, 10 epochs, "
                                          f"trilinear, CTF, SNR {snr}, 32 probes")
    del W
    return out


def conditioning(args, torch, ops, synth):
    """Section 3.1's conditioning analysis: kappa of diag(H) over the ball of
    radius R (nearest interpolation, no CTF, so H is diagonal) for N = 10000
    uniform poses and lam = 1e-8, against the lower bound of Eq. cond number
    p, R = 1, 17, 33, ... on a 512^3 grid."""
    import numpy as np
    h = ops.Handle(torch.cuda.current_device())
    M, N, lam = 512, 10000, 1e-8
    geom = ops.Geometry(M, M // 2 - 1, "nearest", None)
    q = torch.from_numpy(synth.shoemake_quaternions(N, 9100).astype("float32")).cuda()
    rot = h.quat_to_rot(q)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    d, _, _ = h.exact_diag(geom, rot, None, lam, 1.0)
    lo, hi, cnt = h.shell_minmax(d, M // 2)
    e1.record()
    torch.cuda.synchronize()
    lo, hi, cnt = lo.cpu().numpy(), hi.cpu().numpy(), cnt.cpu().numpy()
    k = np.arange(M) - M // 2
    q2 = k[:, None] ** 2 + k[None, :] ** 2
    n2 = np.bincount(np.rint(np.sqrt(q2)).astype(int).ravel(), minlength=M)[: M // 2]
    radii = list(range(1, M // 2 - 1, 16))
    rows = []
    for R in radii:
        kap = float(np.max(hi[: R + 1]) / np.min(lo[: R + 1]))
        p = float(np.sum(n2[: R + 1]) / np.sum(cnt[: R + 1]))
        bound = (N + lam) / (p * N + lam) if 1 / p <= N else None
        rows.append({"R": R, "kappa": kap, "lower_bound": bound})
    del d
    h.close()
    return {"workload": f"{M}^3 grid, {N} uniform poses, nearest, no CTF, lambda {lam}",
            "ms": round(e0.elapsed_time(e1), 3), "by_radius": rows}


def multi_volume(args, torch, ops, synth):
    """Throughput of the multi-volume step, replayed as a CUDA graph: grids
    64/96/128/160 (10k-40k images each, batch 1024 per volume) in one
    autotuned launch; then the same four with the 256^3 problem of 102 400
    images added to the graph (its traversals split into z-slabs)."""
    h = ops.Handle(torch.cuda.current_device())
    specs = [(64, 10240, 200), (96, 20480, 600), (128, 30720, 1000), (160, 40960, 1500)]
    probs, keep = [], []

    def add(M, n_img, blobs, seed):
        cfg = dict(M=M, n_img=n_img, B=1024, interp="trilinear", K=32, df=(1.0, 3.0),
                   snr=0.05, blobs=blobs, seed=seed)
        W = build_workload(cfg, 0, h, torch, ops, synth)
        lam = W["sigma2"]
        alpha = h.threshold_alpha(W["geom"], W["df"], W["n_img"], lam)
        v0 = torch.from_numpy(synth.initial_volume(M, M // 2 - 1, 1.0, 7)).cuda()
        st = ops.SGDState(v0, mode="hutchinson", alpha=alpha, n_probes=32, seed=5)
        probs.append(ops.Problem(W["geom"], st, W["images"], W["quat"], W["df"], 1024, lam,
                                 W["n_img"] / 1024))
        keep.append(W)

    def run(label_volumes):
        bt, bps = h.autotune(probs)
        g = h.multi_step_graph(probs)
        s = torch.cuda.current_stream()
        for _ in range(args.warmup):
            g.launch(s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        steps = max(args.steps, 10)
        for _ in range(steps):
            g.launch(s)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        imgs = 1024 * len(probs) * steps
        g.close()
        return {"volumes": label_volumes, "batch_per_volume": 1024,
                "launch_shape": {"block_threads": bt, "blocks_per_sm": bps},
                "ms_per_step": round(ms / steps, 4), "images_per_s": round(imgs / (ms / 1e3), 1),
                "cuda_graph": True}

    for i, (M, n_img, blobs) in enumerate(specs):
        add(M, n_img, blobs, 7000 + 10 * i)
    out = run([f"{M}^3 x {n} images" for M, n, _ in specs])
    add(256, 102400, 5000, 7040)
    out["with_256"] = run([f"{M}^3 x {n} images" for M, n, _ in specs] +
                          ["256^3 x 102400 images (z-slab launches)"])
    h.close()
    return out


# ---------------------------------------------------------- oracle (CPU) arm
def oracle_sample(cfg, n, seed):
    """A bounded sample of the workload for the FP64 oracle (inputs from the
    generator and the oracle's own forward model)."""
    import numpy as np
    import oracle as O
    from paper_2311_16100_gb300 import synth
    M = cfg["M"]
    r = M // 2 - 1
    ctf = (dict(kv=synth.CTF_KV, cs_mm=synth.CTF_CS_MM, amp=synth.CTF_AMP,
                pixel_A=synth.CTF_PIXEL_A) if cfg["df"] else None)
    v_true = synth.blob_volume(M, cfg["blobs"], seed=cfg["seed"])
    R = O.quat_to_rot(synth.shoemake_quaternions(n, seed + 1)).astype(np.float32)
    df = (synth.defocus_angstrom(n, seed + 2, *cfg["df"]) if cfg["df"] else np.zeros(n)
          ).astype(np.float32)
    clean = O.slice_project(v_true, R, df, M, r, cfg["interp"], ctf)
    m = O.disc_mask(M, r).reshape(M, M)
    sig2 = float(np.mean(np.abs(clean[:, m]) ** 2) / cfg["snr"])
    noise = synth.complex_normal((n, M, M), seed + 3, sig2)
    noise[:, ~m] = 0
    x = (clean + noise).astype(np.complex64)
    v0 = synth.initial_volume(M, r, 1.0, cfg["seed"] + 7)
    return dict(M=M, r=r, ctf=ctf, R=R, df=df, x=x, v0=v0, lam=sig2,
                alpha=O.alpha_threshold(df, M, r, ctf, sig2, scale_alpha=cfg["n_img"] / n))


def time_oracle_step(cfg, S):
    import numpy as np
    import oracle as O
    M = S["M"]
    n = len(S["R"])
    t0 = time.perf_counter()
    O.alg1_step(S["v0"], np.ones((M, M, M)), np.zeros((M, M, M)), 1.0, 1, S["x"], S["R"],
                S["df"], M, S["r"], cfg["interp"], S["ctf"], S["lam"], cfg["n_img"] / n,
                S["alpha"], 0.9, 0.5, "hutchinson", n_probes=cfg["K"], seed=cfg["seed"] + 11)
    return time.perf_counter() - t0


def cpu_cores_used():
    try:
        import numpy as np  # noqa: F401
        return 1           # the oracle's numpy operations are single threaded
    except ImportError:
        return 1


def _oracle_replica(cfg, n, seed, barrier, q):
    """One host core: an independent oracle replica (its own sample), timed
    after all replicas have built their samples."""
    S = oracle_sample(cfg, n, seed)
    barrier.wait(timeout=300)
    t0 = time.perf_counter()
    time_oracle_step(cfg, S)
    q.put((n, t0, time.perf_counter()))


def oracle_all_cores(cfg, n_per_core, cores):
    """The oracle as it stands on every host core: one single-threaded
    replica per core (spawned processes), each one Algorithm-1 step on its own
    sample; images of all replicas / wall time from the common start to the
    last finish."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    q = ctx.Queue()
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    procs = [ctx.Process(target=_oracle_replica,
                         args=(cfg, n_per_core, cfg["seed"] + 500 + 10 * i, barrier, q))
             for i in range(cores)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in procs:
            res.append(q.get(timeout=600))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    for k, v in env_keep.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    n = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return n, wall


def cpu_baseline(cfg, n):
    S = oracle_sample(cfg, n, cfg["seed"] + 500)
    t = time_oracle_step(cfg, S)
    single = {"value": round(n / t, 3), "cores": cpu_cores_used(),
              "sample": f"{n} images, one step, {t:.1f} s"}
    cores = os.cpu_count() or 1
    n_all, wall = oracle_all_cores(cfg, max(1, n // 8), cores)
    return {"value": round(n_all / wall, 3), "unit": "images/s", "cores": cores,
            "kind": "oracle",
            "sample": f"one Algorithm-1 step of the FP64 numpy oracle (literal {cfg['K']}-probe "
                      f"Hutchinson, literal Armijo loop) per host core, {max(1, n // 8)} images "
                      f"each of the {cfg['M']}^3 workload, {cores} single-threaded replicas "
                      f"started together, {wall:.1f} s wall",
            "sample_short": f"FP64 oracle: one literal Algorithm-1 step of "
                            f"{max(1, n // 8)} images per core, {cores} replicas, {wall:.1f} s",
            "single_core": single, "host_cores": cores,
            "operators_single_core": oracle_operators(cfg),
            "config1_alg1_run": oracle_config1_run()}


def oracle_config1_run():
    """The whole 32^3 nearest-interpolation run of the oracle on one core:
    1000 images, batch 100, 5 epochs of Algorithm 1 with 16-probe Hutchinson
    estimates (50 steps); compare with the GPU's time for the same run
    (time_to_rel_err.m32_nearest.hutchinson.total_ms)."""
    import numpy as np
    import oracle as O
    from paper_2311_16100_gb300 import synth
    cfg = CONFIGS["m32"]
    M, B, n_img = cfg["M"], cfg["B"], cfg["n_img"]
    S = oracle_sample(cfg, n_img, cfg["seed"] + 950)
    v, D, Da, eta = S["v0"].astype(np.complex128), np.ones((M, M, M)), np.zeros((M, M, M)), 1.0
    k = 0
    t0 = time.perf_counter()
    for ep in range(5):
        perm = synth.permutation(n_img, cfg["seed"] + 31 + ep)
        for b in range(n_img // B):
            idx = perm[b * B:(b + 1) * B]
            k += 1
            out = O.alg1_step(v, D, Da, eta, k, S["x"][idx], S["R"][idx], S["df"][idx], M,
                              S["r"], cfg["interp"], S["ctf"], S["lam"], n_img / B, S["alpha"],
                              0.9, 0.5, "hutchinson", n_probes=cfg["K"], seed=cfg["seed"] + 11)
            v, D, Da, eta = out["v"], out["D"], out["D_avg"], out["eta"]
    t = time.perf_counter() - t0
    return {"steps": k, "seconds": round(t, 2), "images_per_s": round(k * B / t, 2),
            "cores": 1, "workload": "32^3, 1000 images, batch 100, 5 epochs, nearest, no CTF, "
                                    "16 probes"}


def oracle_operators(cfg):
    """The oracle's loss + gradient and Hutchinson estimate alone, one core:
    16 images of this workload, and 4 images of the 256^3 one."""
    import oracle as O
    out = {}
    for label, c, n in (("%d^3" % cfg["M"], cfg, 16), ("256^3", CONFIGS["m256"], 4)):
        S = oracle_sample(c, n, c["seed"] + 600)
        t0 = time.perf_counter()
        O.loss_grad(S["v0"], S["x"], S["R"], S["df"], c["M"], S["r"], c["interp"], S["ctf"],
                    S["lam"], 1.0)
        t1 = time.perf_counter()
        out[label] = {"loss_grad_images_per_s": round(n / (t1 - t0), 3)}
        if c is cfg:
            t0 = time.perf_counter()
            O.hutchinson_diag(S["R"], S["df"], c["M"], S["r"], c["interp"], S["ctf"], S["lam"],
                              1.0, c["K"], 1, 1)
            t1 = time.perf_counter()
            out[label]["hutchinson_images_per_s"] = round(n / (t1 - t0), 3)
    return out


def run_reference(args, cfg, rank, world):
    if rank != 0:
        return
    n = max(1, min(args.cpu_sample, 8))
    S = oracle_sample(cfg, n, cfg["seed"] + 900)
    for _ in range(args.warmup):
        time_oracle_step(cfg, S)
    ts = [time_oracle_step(cfg, S) for _ in range(args.steps)]
    tot = sum(ts)
    val = n * args.steps / tot
    line = {"metric": METRIC, "value": round(val, 4), "unit": "images/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(args, cfg),
            "cpu_baseline": {"value": round(val, 4), "unit": "images/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"{n} images per step of the {cfg['M']}^3 workload, "
                                       f"one literal Algorithm-1 step each"},
            "e2e": {"value": round(val, 4), "unit": "images/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_json(args, cfg):
    n_img, B = cfg["n_img"], cfg["B"]
    nf, tail = divmod(n_img, B)
    split = f"{nf} x {B}" + (f" + {tail}" if tail else "")
    return {"workload": f"Algorithm-1 step, {cfg['M']}^3 complex64 volume, {n_img} images "
                        f"{cfg['M']}x{cfg['M']} in HBM (batches {split}), {cfg['interp']}, "
                        f"{'CTF' if cfg['df'] else 'no CTF'}, {cfg['K']} probes",
            "global_batch": B * args.gpus,
            "images_in_hbm_per_gpu": n_img, "parallelism": f"replicas{args.gpus}",
            "l2": "inputs > L2: a distinct batch per step"}


ARM_KEYS = {"plain": "plain", "hutchinson": "alg1", "precomputed": "pre", "learned": "learned",
            "exact_diagonal_control": "exact"}


def metric2_summary(tte, learned):
    """Time-to-relative-error races in a few hundred bytes: per workload and
    arm, [final relative error, device ms of the steps to 1e-2 or null], and
    for the arms with a fixed preconditioner built before the first step the
    device ms of that set-up as a third entry, when the race recorded it."""
    sel = [("m32_snr0.1", (tte or {}).get("m32_nearest")),
           ("m64_snr0.05", (tte or {}).get("m64_trilinear_ctf")),
           ("m64_snr10_b4096", (learned or {}).get("time_to_rel_err_64_snr10_b4096"))]
    out = {}
    for key, res in sel:
        if not res:
            continue
        out[key] = {}
        for a, short in ARM_KEYS.items():
            if a in res:
                ms = res[a]["ms_to_rel_err"]["0.01"]
                out[key][short] = [round(res[a]["final_rel_err"], 4),
                                   None if ms is None else round(ms, 1)]
        for a, ms in (res.get("setup_ms") or {}).items():
            short = ARM_KEYS.get(a)
            if short in out[key]:
                out[key][short].append(round(ms, 1))
    return out or None


def contract_line(args, cfg, world, r, cpu=None, metric2=None):
    """The benchmark's record: the last line bench.py prints, a few KB at
    most.  ``r`` is run_gpu's result; ``cpu`` the oracle baseline; ``metric2``
    metric2_summary's result."""
    ms_step = r["ms"] / args.steps
    value = world * r["timed_images"] / (r["ms"] / 1e3)
    e2e = None
    if r.get("e2e"):
        e = r["e2e"]
        e2e = {k: (round(e[k], 1) if isinstance(e[k], float) else e[k])
               for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step",
                         "full_images_value", "direct_value") if k in e}
        e2e["api"] = "cs_precond_sgd_step_host_disc"
        if "h2d_copy_only" in e:
            e2e["h2d_copy_only_GB_per_s"] = e["h2d_copy_only"]["GB_per_s"]
    cpu_line = None
    if cpu:
        cpu_line = {k: cpu[k] for k in ("value", "unit", "cores", "kind")}
        cpu_line["sample"] = cpu.get("sample_short", cpu["sample"])
        if "single_core" in cpu:
            cpu_line["single_core_value"] = cpu["single_core"]["value"]
    line = {"metric": METRIC, "value": round(value, 1), "unit": "images/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_json(args, cfg),
            "roofline": r["roofline"],
            "roofline_l2_reductions": ({k: v for k, v in r["red_roofline"].items()
                                        if k != "peak_source"}
                                       if r.get("red_roofline") else None),
            "e2e": e2e, "gpu_launches": r["launches"],
            "clocks": ({k: r["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}
                       if r.get("clocks") else None),
            "cpu_baseline": cpu_line, "phases_ms_per_step": r.get("phases"),
            "metric2": metric2}
    return line


def emit_aux(name, payload):
    """An auxiliary leg's full result, on its own line before the record."""
    print(json.dumps({"aux": name, "result": payload}), flush=True)


def main():
    args = parse()
    cfg = workload_config(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return
    if args.mlp_only:
        mlp_only(args)
        return
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r = run_gpu(args, cfg, rank, world)
    if rank == 0:
        emit_aux("step_details", {k: r[k] for k in ("phases", "e2e", "graph", "loss_grad_only",
                                                    "red_roofline", "scalars")})
        tte = learned = cpu = None
        if world == 1 and not args.no_metric2:
            from paper_2311_16100_gb300 import ops, synth
            h2 = ops.Handle(torch.cuda.current_device())
            tte = {k: time_to_error(c, torch, ops, synth, h2) for k, c in TTE_CONFIGS.items()}
            h2.close()
            emit_aux("time_to_rel_err", tte)
        if world == 1 and not args.no_learned:
            from paper_2311_16100_gb300 import ops, synth
            learned = learned_leg(args, torch, ops, synth)
            emit_aux("learned_preconditioner", learned)
        if world == 1 and not args.no_metric2:
            from paper_2311_16100_gb300 import ops, synth
            emit_aux("conditioning", conditioning(args, torch, ops, synth))
        if world == 1 and not args.no_multi:
            from paper_2311_16100_gb300 import ops, synth
            emit_aux("multi_volume", multi_volume(args, torch, ops, synth))
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(cfg, args.cpu_sample)
            emit_aux("cpu_baseline", cpu)
        line = contract_line(args, cfg, world, r, cpu, metric2_summary(tte, learned))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
