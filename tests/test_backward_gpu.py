"""GPU backward (mgs_render_backward through torch.autograd) against the
oracle gradient (oracle/grad.py, FP64 autograd of the pinned oracle).

Gradients are compared per parameter kind: max |GPU - oracle| <= tol * max
|oracle| of that kind (FP32 accumulation over many pixels against FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import grad as og
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu

COLS = {"mu": (0, 3), "s": (3, 6), "q": (6, 10), "o": (10, 11), "Y": (11, 23)}


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield r
    r.close()


def _gpu_grads(R, attrs, cam, dL, mlp=None, use_mlp=False, res=False, bg=(0.0, 0.0, 0.0)):
    from paper_2603_11531_gb300 import autograd as ag
    a = torch.from_numpy(attrs.astype(np.float32)).cuda().requires_grad_(True)
    mt = None
    if mlp is not None and use_mlp:
        w = lambda b: torch.from_numpy(synth.bf16_bits_to_f32(b).copy()).cuda().requires_grad_(True)
        f = lambda x: torch.from_numpy(np.asarray(x, np.float32).copy()).cuda().requires_grad_(True)
        mt = (w(mlp.w1), f(mlp.b1), w(mlp.w2), f(mlp.b2), w(mlp.w3), f(mlp.b3))
    img = ag.render(R, a, cam, mt, use_mlp=use_mlp, rgb_residual=res, bg=bg)
    (img * torch.from_numpy(dL.astype(np.float32)).cuda()).sum().backward()
    out = {"attrs": a.grad.cpu().numpy().astype(np.float64)}
    if mt is not None:
        for k, t in zip(("w1", "b1", "w2", "b2", "w3", "b3"), mt):
            out[k] = t.grad.cpu().numpy().astype(np.float64)
    return out, img.detach().cpu().numpy()


def _ref_grads(attrs, cam, dL, mlp=None, use_mlp=False, res=False, bg=(0.0, 0.0, 0.0)):
    st = og.discrete_structure(attrs, cam, mlp, use_mlp, res)
    p = og.params_from_scene(attrs, mlp if use_mlp else None)
    g = og.loss_grad(p, cam, st, dL, use_mlp=use_mlp, rgb_residual=res, bg=bg)
    return {k: v.numpy() for k, v in g.items()}


def _compare(gpu, ref, tol, kinds=COLS, mlp_keys=()):
    for name, (c0, c1) in kinds.items():
        got = gpu["attrs"][:, c0:c1].reshape(ref[name].shape)
        scale = np.abs(ref[name]).max()
        err = np.abs(got - ref[name]).max()
        assert err <= tol * scale + 1e-9, (name, err, scale)
    for k in mlp_keys:
        scale = np.abs(ref[k]).max()
        err = np.abs(gpu[k] - ref[k]).max()
        assert err <= tol * scale + 1e-9, (k, err, scale)


def test_backward_plain_fp32_matches_oracle_gradient(R):
    s = synth.uniform_scene(300, seed=5, precision="fp32")
    cam = synth.look_at((0.2, -0.1, -2.6), (0, 0, 0), 48, 40, 60.0)
    dL = np.random.default_rng(0).normal(size=(40, 48, 3))
    bg = (0.3, 0.2, 0.1)
    gpu, img = _gpu_grads(R, s.attrs, cam, dL, bg=bg)
    ref = _ref_grads(s.attrs, cam, dL, bg=bg)
    _compare(gpu, ref, tol=2e-3)
    assert np.all(gpu["attrs"][:, 23] == 0)


def test_backward_mlp_residual_matches_oracle_gradient(R):
    s = synth.uniform_scene(400, seed=6, precision="fp32")
    s.mlp = synth.random_mlp(8)
    cam = synth.look_at((-0.3, 0.2, -2.8), (0, 0, 0), 64, 48, 60.0)
    dL = np.random.default_rng(1).normal(size=(48, 64, 3))
    gpu, img = _gpu_grads(R, s.attrs, cam, dL, s.mlp, use_mlp=True, res=True)
    ref = _ref_grads(s.attrs, cam, dL, s.mlp, use_mlp=True, res=True)
    kinds = dict(COLS)
    kinds.pop("o")        # the stored opacity is unused with the MLP
    _compare(gpu, ref, tol=5e-3, kinds=kinds, mlp_keys=("w1", "b1", "w2", "b2", "w3", "b3"))
    assert np.all(gpu["attrs"][:, 10] == 0)


def test_backward_fp16_attributes(R):
    s = synth.unbounded_scene(5000, seed=9, precision="fp16")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 96, 64, 60.0)[2]
    dL = np.random.default_rng(2).normal(size=(64, 96, 3))
    gpu, _ = _gpu_grads(R, s.attrs, cam, dL)
    ref = _ref_grads(s.attrs, cam, dL)
    _compare(gpu, ref, tol=2e-3)


@pytest.mark.slow
@pytest.mark.parametrize("use_mlp", [True, False])
def test_backward_300k_directional_derivative(R, use_mlp):
    """The backward workload (300k Gaussians, FP32, 1296x840, L1 loss against a
    seeded target): the GPU gradient predicts the change of the GPU loss along
    a random direction in which the forward is smooth -- the MLP head bias
    (FP32, after the last BF16-rounded activation) with the MLP, SH and
    opacity of every Gaussian without it (geometry would move the inclusion
    boundaries; the MLP's BF16-rounded inputs make it piecewise constant)."""
    from paper_2603_11531_gb300 import autograd as ag
    scene, cam, target = synth.workload_backward_300k()
    a = torch.from_numpy(scene.attrs).cuda().requires_grad_(True)
    w = lambda b: torch.from_numpy(synth.bf16_bits_to_f32(b).copy()).cuda()
    f = lambda x: torch.from_numpy(np.asarray(x, np.float32).copy()).cuda()
    mlp = (w(scene.mlp.w1), f(scene.mlp.b1), w(scene.mlp.w2), f(scene.mlp.b2),
           w(scene.mlp.w3), f(scene.mlp.b3).requires_grad_(True)) if use_mlp else None
    tgt = torch.from_numpy(target).cuda().double()

    def loss(attrs, m):
        img = ag.render(R, attrs, cam, m, use_mlp=use_mlp)
        return (img.double() - tgt).abs().sum()

    loss(a, mlp).backward()
    assert torch.isfinite(a.grad).all()
    gen = torch.Generator(device="cuda").manual_seed(3)
    eps = 1e-3
    if use_mlp:
        v = torch.randn(5, device="cuda", generator=gen)
        pred = float((mlp[5].grad.double() * v.double()).sum())
        with torch.no_grad():
            mp = mlp[:5] + (mlp[5] + eps * v,)
            mm = mlp[:5] + (mlp[5] - eps * v,)
            fd = float(loss(a, mp) - loss(a, mm)) / (2 * eps)
    else:
        v = torch.zeros_like(a)
        v[:, 10:23] = torch.randn(scene.n, 13, device="cuda", generator=gen)
        v[:, 10] *= 0.1
        pred = float((a.grad.double() * v.double()).sum())
        with torch.no_grad():
            fd = float(loss(a + eps * v, None) - loss(a - eps * v, None)) / (2 * eps)
    assert abs(fd - pred) <= 0.02 * abs(pred), (fd, pred)


def _render_np(m, R, h, cam, opts, aux=None, count=None):
    H, W = cam.height, cam.width
    rgb = torch.empty((H, W, 3), device="cuda")
    m.mgs_render_checked(R.ws, h, cam, opts, rgb, aux, count)
    return rgb.double()


def test_backward_finite_differences_512_at_64x64(R):
    """The backward workload's first 512 Gaussians (unbounded distribution,
    FP32) at 64x64: the GPU adjoint against central differences of the GPU
    forward, for means, scales, quaternions, opacities and SH coefficients
    of sampled Gaussians (plain mode).  The loss weights only the pixels near
    the perturbed Gaussian (dL random there, 0 elsewhere), so the FP32
    rounding of unrelated pixels stays out of the difference; a parameter
    whose +-h changes any pixel's inclusion count is skipped (the inclusion
    test is piecewise constant)."""
    import paper_2603_11531_gb300 as m
    scene, _, _ = synth.workload_backward_300k()
    attrs = np.ascontiguousarray(scene.attrs[:512], np.float32)
    cam = synth.orbit_cameras(1, 8.0, 1.0, 64, 64, 60.0)[0]
    H, W = cam.height, cam.width
    g = oracle.preprocess(attrs, cam)
    vis = np.flatnonzero(g["visible"] == 1)
    rng = np.random.default_rng(7)
    pick = rng.choice(vis, size=min(20, len(vis)), replace=False)
    opts = m.render_opts()
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    checked = skipped = 0
    comps = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 15, 19]
    for i in pick:
        c = g["conic"][i]
        dx, dy = xx - g["mean"][i][0], yy - g["mean"][i][1]
        near = c[0] * dx * dx + 2 * c[1] * dx * dy + c[2] * dy * dy <= 12.0
        dL = np.zeros((H, W, 3))
        dL[near] = rng.normal(size=(int(near.sum()), 3))
        dLt = torch.from_numpy(dL).cuda()
        h0 = R.load_scene(attrs)
        try:
            aux = torch.empty((5, H, W), device="cuda")
            cnt0 = torch.empty((H, W), dtype=torch.int32, device="cuda")
            _render_np(m, R, h0, cam, opts, aux, cnt0)
            d_attrs = torch.empty((512, 24), device="cuda")
            m.mgs_render_backward(R.ws, h0, cam, opts, dLt.float(), aux, d_attrs)
            grad = d_attrs.cpu().numpy().astype(np.float64)
        finally:
            R.unload_scene(h0)
        for k in comps:
            x = float(attrs[i, k])
            # steps large enough that the loss change stands well above the
            # FP32 rounding of the footprint's pixels, small against the
            # Gaussian's extent (means are world units, about 7 px per unit)
            step = 1e-2 * max(abs(x), 0.05) if 3 <= k < 6 else 1e-2
            imgs, same = [], True
            for sgn in (1.0, -1.0):
                a = attrs.copy()
                a[i, k] = np.float32(x + sgn * step)
                hs = R.load_scene(a)
                try:
                    cnt = torch.empty((H, W), dtype=torch.int32, device="cuda")
                    imgs.append(_render_np(m, R, hs, cam, opts, None, cnt))
                    same &= bool(torch.equal(cnt, cnt0))
                finally:
                    R.unload_scene(hs)
            # the step actually taken in FP32
            hstep = (float(np.float32(x + step)) - float(np.float32(x - step))) / 2.0
            if not same:
                skipped += 1
                continue
            fd = float((dLt * (imgs[0] - imgs[1])).sum()) / (2.0 * hstep)
            gk = grad[i, k]
            # FP32 rounding of the two images (2^-23 of values below 2, over
            # the weighted pixels) bounds the difference quotient's noise
            noise = 4.0 * 2.0 ** -23 * float(np.sqrt((dL ** 2).sum())) / (2.0 * hstep)
            assert abs(fd - gk) <= 0.03 * abs(gk) + noise, (int(i), k, fd, gk, noise)
            checked += 1
    assert checked >= 0.8 * (checked + skipped) and checked > 100, (checked, skipped)


def test_backward_finite_differences_mlp_head_bias_64x64(R):
    """With the MLP (FP32 attributes, BF16 MLP): the gradient of the head
    biases b3 (FP32, after the last BF16-rounded activation, so the forward is
    smooth in them) against central differences of the GPU forward, on the
    backward workload's first 512 Gaussians at 64x64."""
    from paper_2603_11531_gb300 import autograd as ag
    scene, _, _ = synth.workload_backward_300k()
    attrs = torch.from_numpy(np.ascontiguousarray(scene.attrs[:512], np.float32)).cuda()
    cam = synth.orbit_cameras(1, 8.0, 1.0, 64, 64, 60.0)[0]
    w = lambda b: torch.from_numpy(synth.bf16_bits_to_f32(b).copy()).cuda()
    f = lambda x: torch.from_numpy(np.asarray(x, np.float32).copy()).cuda()
    b3 = f(scene.mlp.b3).requires_grad_(True)
    head = (w(scene.mlp.w1), f(scene.mlp.b1), w(scene.mlp.w2), f(scene.mlp.b2), w(scene.mlp.w3))
    dL = torch.from_numpy(np.random.default_rng(8).normal(size=(64, 64, 3))).cuda()
    img = ag.render(R, attrs, cam, head + (b3,), use_mlp=True, rgb_residual=True)
    (img.double() * dL).sum().backward()
    grad = b3.grad.double().cpu().numpy()
    eps = 1e-2
    for k in range(5):
        with torch.no_grad():
            e = torch.zeros(5, device="cuda")
            e[k] = eps
            lp = (ag.render(R, attrs, cam, head + (b3 + e,), use_mlp=True, rgb_residual=True).double()
                  * dL).sum()
            lm = (ag.render(R, attrs, cam, head + (b3 - e,), use_mlp=True, rgb_residual=True).double()
                  * dL).sum()
        fd = float(lp - lm) / (2 * eps)
        assert abs(fd - grad[k]) <= 0.02 * abs(grad[k]) + 1e-3, (k, fd, grad[k])


@pytest.mark.slow
def test_backward_30k_320x240_mlp_matches_oracle_gradient(R, error_report):
    """30k Gaussians of the unbounded distribution (FP32, BF16 MLP with the
    colour residual) at 320x240, so that many pixels and tiles accumulate
    into the same Gaussians' gradient records (atomics under contention):
    means, scales, quaternions and SH rows and every MLP weight against the
    FP64 oracle gradient."""
    s = synth.unbounded_scene(30000, seed=31, precision="fp32")
    s.mlp = synth.random_mlp(32)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 320, 240, 60.0)[3]
    dL = np.random.default_rng(4).normal(size=(240, 320, 3))
    gpu, _ = _gpu_grads(R, s.attrs, cam, dL, s.mlp, use_mlp=True, res=True)
    ref = _ref_grads(s.attrs, cam, dL, s.mlp, use_mlp=True, res=True)
    kinds = dict(COLS)
    kinds.pop("o")
    report = {}
    for name, (c0, c1) in kinds.items():
        got = gpu["attrs"][:, c0:c1].reshape(ref[name].shape)
        report[name] = float(np.abs(got - ref[name]).max() / np.abs(ref[name]).max())
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        report[k] = float(np.abs(gpu[k] - ref[k]).max() / np.abs(ref[k]).max())
    error_report["backward_30k_320x240_mlp_relative_to_max_per_kind"] = report
    _compare(gpu, ref, tol=5e-3, kinds=kinds, mlp_keys=("w1", "b1", "w2", "b2", "w3", "b3"))
