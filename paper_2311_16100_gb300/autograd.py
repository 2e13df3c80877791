"""torch.autograd.Function for the Fourier-slice operator.

forward:  images = C P v   (cs_slice_project; Definition 2.1, Eq. fwd model)
backward: grad_v = P^* C grad_images   (cs_backproject_adjoint)

For a real-valued loss, PyTorch's complex gradients are dL/dRe + i dL/dIm,
and the operator v -> C P v has real coefficients, so the vector-Jacobian
product is the adjoint P^* C applied to the incoming gradient.  The paper
obtains Hessian-vector products through automatic differentiation
(Section 3.2); with this Function, torch's autograd runs the library's
adjoint kernel for that step.  Rotations and defocus receive no gradient.
"""
from __future__ import annotations

import torch

from .ops import Geometry, Handle

_handles: dict[int, Handle] = {}


def default_handle(device: torch.device | int | None = None) -> Handle:
    """One library handle per CUDA device, created on first use."""
    if device is None:
        idx = torch.cuda.current_device()
    elif isinstance(device, torch.device):
        idx = device.index if device.index is not None else torch.cuda.current_device()
    else:
        idx = int(device)
    h = _handles.get(idx)
    if h is None:
        h = Handle(idx)
        _handles[idx] = h
    return h


class SliceProject(torch.autograd.Function):
    """images[B][M][M] = C_i P_i v for complex64 v[M][M][M]."""

    @staticmethod
    def forward(ctx, vol, rot, defocus, geom: Geometry, handle: Handle | None = None):
        h = handle or default_handle(vol.device)
        vol_c = vol.detach().contiguous()
        out = h.slice_project(geom, vol_c, rot.contiguous(),
                              defocus.contiguous() if defocus is not None else None)
        ctx.save_for_backward(rot, defocus if defocus is not None else torch.empty(0))
        ctx.geom = geom
        ctx.handle = h
        ctx.has_defocus = defocus is not None
        ctx.M = vol.shape[0]
        return out

    @staticmethod
    def backward(ctx, grad_out):
        rot, defocus = ctx.saved_tensors
        grad_vol = None
        if ctx.needs_input_grad[0]:
            M = ctx.M
            grad_vol = torch.zeros((M, M, M), dtype=torch.complex64, device=grad_out.device)
            ctx.handle.backproject_adjoint(ctx.geom, grad_out.contiguous(), rot.contiguous(),
                                           defocus.contiguous() if ctx.has_defocus else None,
                                           1.0, vol_accum=grad_vol)
        return grad_vol, None, None, None, None


def slice_project(vol, rot, defocus, geom: Geometry, handle: Handle | None = None):
    """Differentiable C P v (see SliceProject)."""
    return SliceProject.apply(vol, rot, defocus, geom, handle)
