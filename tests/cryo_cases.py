"""Seeded test cases shared by the parity tests.

Inputs come from the synthetic generator; images are formed by the FP64
oracle's forward model plus complex Gaussian noise, then rounded to the
single-precision values the GPU receives.  The oracle is always evaluated
on exactly those rounded values.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2311_16100_gb300 import synth

CTF_DICT = dict(kv=synth.CTF_KV, cs_mm=synth.CTF_CS_MM, amp=synth.CTF_AMP,
                pixel_A=synth.CTF_PIXEL_A)


class Case:
    def __init__(self, M, B, interp="trilinear", ctf=True, seed=0, snr=0.1, r_max=None,
                 n_blobs=None, df_range=(1.0, 3.0)):
        self.M, self.B, self.interp = M, B, interp
        self.r_max = M // 2 - 1 if r_max is None else r_max
        self.ctf = CTF_DICT if ctf else None
        self.vol = synth.blob_volume(M, n_blobs=n_blobs, seed=seed)            # complex64
        self.quat = synth.shoemake_quaternions(B, seed + 1)
        self.R = O.quat_to_rot(self.quat).astype(np.float32)
        self.df = synth.defocus_angstrom(B, seed + 2, *df_range).astype(np.float32)
        clean = O.slice_project(self.vol, self.R, self.df, M, self.r_max, interp, self.ctf)
        m = O.disc_mask(M, self.r_max).reshape(M, M)
        sig2 = np.mean(np.abs(clean[:, m]) ** 2) / snr if B else 1.0
        self.sigma2 = float(sig2)
        noise = synth.complex_normal((B, M, M), seed + 3, sig2)
        noise[:, ~m] = 0
        self.images = (clean + noise).astype(np.complex64)

    # oracle keyword arguments
    def geo(self):
        return dict(M=self.M, r_max=self.r_max, interp=self.interp, ctf=self.ctf)

    def gpu_geometry(self):
        from paper_2311_16100_gb300.ops import CTF, Geometry
        return Geometry(self.M, self.r_max, self.interp, CTF() if self.ctf else None)

    def to_gpu(self):
        import torch
        d = torch.device("cuda")
        return dict(vol=torch.from_numpy(self.vol).to(d),
                    images=torch.from_numpy(self.images).to(d),
                    rot=torch.from_numpy(self.R).to(d).contiguous(),
                    df=torch.from_numpy(self.df).to(d),
                    quat=torch.from_numpy(self.quat.astype(np.float32)).to(d))


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
