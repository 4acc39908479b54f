"""Oracle gradient of the sort-free renderer: a differentiable FP64 restatement.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The forward below
restates, in plain PyTorch CPU FP64 ops, the same computation as the C oracle
(``mgs_oracle.c``): App. B projection and EWA covariance, Sec. 3.2 degree-1
SH colour, Eq. 4 MLP, Eq. 3 weight and the Eq. 2 composite.  The discrete
parts -- which Gaussians are visible, the tile rectangles and the per-pixel
inclusion test (the FP32 contract) -- are taken from the C oracle as a fixed
list of included (pixel, Gaussian) pairs; their derivative is zero almost
everywhere.  ``torch.autograd`` (a library primitive) then gives the exact
gradient of this FP64 definition.  The BF16 rounding of the MLP's tensor-core
inputs is applied in the forward and passed straight through in the backward
(its derivative is zero almost everywhere, so the identity is the usual
convention); ``round_bf16=False`` gives the unrounded function used for
finite-difference checks.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import preprocess, bin_tiles, included_pairs

SH_C0 = 0.5 / math.sqrt(math.pi)
SH_C1 = math.sqrt(3.0) * 0.5 / math.sqrt(math.pi)


class _BF16Round(torch.autograd.Function):
    """Nearest BF16 (ties to even) in the forward, identity in the backward."""

    @staticmethod
    def forward(ctx, x):
        return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g


def _bf16(x, on: bool):
    return _BF16Round.apply(x) if on else x


def params_from_scene(attrs: np.ndarray, mlp=None) -> dict:
    """FP64 leaf tensors (requires_grad) for every differentiable input."""
    a = torch.from_numpy(np.asarray(attrs).astype(np.float64))
    p = {"mu": a[:, 0:3].clone(), "s": a[:, 3:6].clone(), "q": a[:, 6:10].clone(),
         "o": a[:, 10].clone(), "Y": a[:, 11:23].clone()}
    if mlp is not None:
        from_bits = lambda b: torch.from_numpy(
            (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64))
        p.update(w1=from_bits(mlp.w1), b1=torch.from_numpy(mlp.b1.astype(np.float64)),
                 w2=from_bits(mlp.w2), b2=torch.from_numpy(mlp.b2.astype(np.float64)),
                 w3=from_bits(mlp.w3), b3=torch.from_numpy(mlp.b3.astype(np.float64)))
    for v in p.values():
        v.requires_grad_(True)
    return p


def discrete_structure(attrs, cam, mlp=None, use_mlp=False, rgb_residual=False):
    """Visible set and included pairs from the C oracle (FP32 contract)."""
    g = preprocess(attrs, cam, mlp, use_mlp, rgb_residual)
    off, gids = bin_tiles(g, cam.width, cam.height)
    pix, gid = included_pairs(g, off, gids, cam.width, cam.height)
    return {"gauss": g, "pix": torch.from_numpy(pix), "gid": torch.from_numpy(gid.astype(np.int64))}


def _rotation(qh):
    w, x, y, z = qh[:, 0], qh[:, 1], qh[:, 2], qh[:, 3]
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=1)
    return R.reshape(-1, 3, 3)


def render(p: dict, cam, struct: dict, use_mlp=False, rgb_residual=False, bg=(0.0, 0.0, 0.0),
           round_bf16=True):
    """FP64 image (H, W, 3) as a differentiable function of the leaves in p."""
    W = torch.tensor(np.asarray(cam.R, np.float32).reshape(3, 3).astype(np.float64))
    tc = torch.tensor(np.asarray(cam.t, np.float32).astype(np.float64))
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    cx, cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    H, Wd = int(cam.height), int(cam.width)
    mu, s, q, Y = p["mu"], p["s"], p["q"], p["Y"]

    qh = q / q.norm(dim=1, keepdim=True)
    R = _rotation(qh)
    t = mu @ W.T + tc
    S3 = R @ torch.diag_embed(s * s) @ R.transpose(1, 2)
    SC = W @ S3 @ W.T
    limx = 1.3 * (0.5 * Wd / fx)
    limy = 1.3 * (0.5 * H / fy)
    u, v = t[:, 0] / t[:, 2], t[:, 1] / t[:, 2]
    uc, vc = u.clamp(-limx, limx), v.clamp(-limy, limy)
    z0 = torch.zeros_like(u)
    J = torch.stack([torch.stack([fx / t[:, 2], z0, -fx * uc / t[:, 2]], 1),
                     torch.stack([z0, fy / t[:, 2], -fy * vc / t[:, 2]], 1)], 1)
    S2 = J @ SC @ J.transpose(1, 2)
    a = S2[:, 0, 0] + 0.3
    b = 0.5 * (S2[:, 0, 1] + S2[:, 1, 0])
    c = S2[:, 1, 1] + 0.3
    det = a * c - b * b
    A, B, C = c / det, -b / det, a / det
    mx, my = fx * u + cx, fy * v + cy

    centre = -(W.T @ tc)
    d = mu - centre
    P = d / d.norm(dim=1, keepdim=True)

    phi = torch.ones_like(u)
    o = p["o"]
    res = None
    if use_mlp:
        x = torch.cat([P, s, qh, Y], dim=1)
        h1 = _bf16(torch.relu(_bf16(x, round_bf16) @ p["w1"].T + p["b1"]), round_bf16)
        h2 = _bf16(torch.relu(h1 @ p["w2"].T + p["b2"]), round_bf16)
        y = h2 @ p["w3"].T + p["b3"]
        phi = torch.relu(y[:, 0])
        o = torch.sigmoid(y[:, 1])
        res = y[:, 2:5]
    Yc = Y.reshape(-1, 4, 3)
    base = (SH_C0 * Yc[:, 0] - SH_C1 * P[:, 1:2] * Yc[:, 1] + SH_C1 * P[:, 2:3] * Yc[:, 2]
            - SH_C1 * P[:, 0:1] * Yc[:, 3] + 0.5)
    if use_mlp and rgb_residual:
        base = base + res
    rgb = torch.clamp(base, min=0.0)
    smax = s.max(dim=1).values
    dz = t[:, 2]
    w = phi * phi + phi / (dz * dz) + torch.exp(smax / dz)

    pix, gid = struct["pix"], struct["gid"]
    py = torch.div(pix, Wd, rounding_mode="floor").to(torch.float64)
    px = (pix % Wd).to(torch.float64)
    dx = px + 0.5 - mx[gid]
    dy = py + 0.5 - my[gid]
    qq = A[gid] * dx * dx + 2.0 * B[gid] * dx * dy + C[gid] * dy * dy
    alpha = torch.clamp(o[gid] * torch.exp(-0.5 * qq), max=0.99)
    aw = alpha * w[gid]
    npx = H * Wd
    Aacc = torch.zeros(npx, 3, dtype=torch.float64).index_add(0, pix, rgb[gid] * aw[:, None])
    Bacc = torch.zeros(npx, dtype=torch.float64).index_add(0, pix, aw)
    logT = torch.zeros(npx, dtype=torch.float64).index_add(0, pix, torch.log1p(-alpha))
    T = torch.exp(logT)
    bgv = torch.tensor(bg, dtype=torch.float64)
    safeB = torch.where(Bacc > 0, Bacc, torch.ones_like(Bacc))
    fg = torch.where((Bacc > 0)[:, None], (1 - T)[:, None] * Aacc / safeB[:, None],
                     torch.zeros_like(Aacc))
    out = fg + T[:, None] * bgv
    return out.reshape(H, Wd, 3)


def loss_grad(p: dict, cam, struct: dict, dL_dC: np.ndarray, **kw) -> dict:
    """Gradient of L = sum(dL_dC * C) with respect to every leaf (FP64)."""
    for v in p.values():
        if v.grad is not None:
            v.grad = None
    img = render(p, cam, struct, **kw)
    L = (img * torch.from_numpy(np.asarray(dL_dC, np.float64))).sum()
    L.backward()
    return {k: v.grad.detach().clone() if v.grad is not None else torch.zeros_like(v)
            for k, v in p.items()}
