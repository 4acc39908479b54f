"""torch.autograd.Function around mgs_render / mgs_render_backward.

Training-style use: Gaussian attributes (N, 24) and, optionally, the MLP
parameters are CUDA tensors that require grad.  Every step of the forward and
backward runs in the library's kernels; this module only moves tensors across
the C-ABI (the MLP weights are rounded to BF16 bit patterns for the tensor
cores on the way in).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (MLP_GRAD_SIZE, Renderer, mgs_load_scene, mgs_render_checked, mgs_render_backward,
               mgs_unload_scene, render_opts)
from .synth import MLPWeights, f32_to_bf16_bits

_SHAPES = (("w1", (64, 22)), ("b1", (64,)), ("w2", (64, 64)), ("b2", (64,)),
           ("w3", (5, 64)), ("b3", (5,)))


def _mlp_from_tensors(ts) -> MLPWeights:
    arr = [t.detach().float().cpu().numpy() for t in ts]
    return MLPWeights(f32_to_bf16_bits(arr[0]), arr[1].astype(np.float32),
                      f32_to_bf16_bits(arr[2]), arr[3].astype(np.float32),
                      f32_to_bf16_bits(arr[4]), arr[5].astype(np.float32))


class RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, cam, opts, attrs, *mlp):
        mlpw = _mlp_from_tensors(mlp) if mlp else None
        scene = mgs_load_scene(renderer.ctx, attrs.detach().contiguous(), mlpw)
        H, W = int(cam.height), int(cam.width)
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=attrs.device)
        aux = torch.empty((5, H, W), dtype=torch.float32, device=attrs.device)
        try:
            mgs_render_checked(renderer.ws, scene, cam, opts, rgb, aux)
        except Exception:
            mgs_unload_scene(scene)
            raise
        ctx.renderer, ctx.cam, ctx.opts, ctx.scene = renderer, cam, opts, scene
        ctx.n_mlp = len(mlp)
        ctx.attrs_shape, ctx.attrs_dtype = attrs.shape, attrs.dtype
        ctx.save_for_backward(aux)
        return rgb

    @staticmethod
    def backward(ctx, g):
        (aux,) = ctx.saved_tensors
        dev = aux.device
        d_attrs = torch.empty(ctx.attrs_shape, dtype=torch.float32, device=dev)
        d_mlp = torch.empty(MLP_GRAD_SIZE, dtype=torch.float32, device=dev) if ctx.n_mlp else None
        try:
            mgs_render_backward(ctx.renderer.ws, ctx.scene, ctx.cam, ctx.opts, g.contiguous(), aux,
                                d_attrs, d_mlp)
            torch.cuda.synchronize(dev)
        finally:
            mgs_unload_scene(ctx.scene)
        grads = [None, None, None, d_attrs.to(ctx.attrs_dtype)]
        if ctx.n_mlp:
            off = 0
            for _, shp in _SHAPES:
                k = int(np.prod(shp))
                grads.append(d_mlp[off:off + k].view(shp))
                off += k
        return tuple(grads)


def render(renderer: Renderer, attrs: torch.Tensor, cam, mlp: tuple | None = None,
           use_mlp: bool = False, rgb_residual: bool = False, bg=(0.0, 0.0, 0.0)):
    """Differentiable render: returns the (H, W, 3) image; gradients flow to
    `attrs` and, with use_mlp, to the six MLP tensors (w1, b1, w2, b2, w3, b3)."""
    opts = render_opts(use_mlp, rgb_residual, bg)
    if use_mlp:
        if mlp is None or len(mlp) != 6:
            raise ValueError("use_mlp needs the six MLP tensors")
        return RenderFn.apply(renderer, cam, opts, attrs, *mlp)
    return RenderFn.apply(renderer, cam, opts, attrs)
