"""torch.autograd wrappers of LDNI volume and sample depths.

Forward: sample the mesh (exact two-pass) and evaluate; backward: the
library's adjoint kernels (ldni_volume_grad, ldni_depth_vjp) with the
crossing set of the forward pass held fixed.
"""
from __future__ import annotations

import torch

from . import ldni as _L


class LDNIVolume(torch.autograd.Function):
    """volume = LDNIVolume.apply(verts, tris, grid, axis) for one image
    (axis 0..2), or the mean of the three images' volumes for axis 'all'."""

    @staticmethod
    def forward(ctx, verts, tris, grid, axis):
        v = verts.detach().to("cuda", torch.float32).contiguous()
        t = tris.to("cuda", torch.int32).contiguous()
        layers = _L.sample(v, t, grid, axis)
        layers = layers if isinstance(layers, list) else [layers]
        vols = [_L.volume(L) for L in layers]
        ctx.save_for_backward(v, t)
        ctx.layers = layers
        return torch.tensor(sum(vols) / len(vols), dtype=torch.float64, device="cuda")

    @staticmethod
    def backward(ctx, g):
        v, t = ctx.saved_tensors
        grad = torch.zeros(v.shape[0], 3, dtype=torch.float32, device="cuda")
        w = float(g.item()) / len(ctx.layers)
        for L in ctx.layers:
            _L.volume_grad(v, t, L, w, grad)
        return grad.to(torch.float64 if g.dtype == torch.float64 else grad.dtype), None, None, None


class LDNIDepths(torch.autograd.Function):
    """depths = LDNIDepths.apply(verts, tris, grid, axis): the sample depths
    of one image in CSR order (offsets available as the .layers attribute of
    the returned tensor's grad_fn context)."""

    @staticmethod
    def forward(ctx, verts, tris, grid, axis):
        v = verts.detach().to("cuda", torch.float32).contiguous()
        t = tris.to("cuda", torch.int32).contiguous()
        L = _L.sample(v, t, grid, int(axis))
        ctx.save_for_backward(v, t)
        ctx.L = L
        return L.depth[:L.n].clone()

    @staticmethod
    def backward(ctx, g):
        v, t = ctx.saved_tensors
        grad = _L.depth_vjp(v, t, ctx.L, g.to(torch.float32))
        return grad, None, None, None
