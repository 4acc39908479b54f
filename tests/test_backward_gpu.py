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
