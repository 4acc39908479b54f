"""Pins of the oracle gradient (oracle/grad.py) -- CPU only.

* its forward equals the C oracle's image (so the gradient is the gradient of
  the pinned oracle, with the discrete inclusion structure held fixed);
* its autograd gradient equals central finite differences of the C oracle's
  FP64 forward (plain mode) for randomly chosen parameters of every kind,
  skipping a parameter only if its perturbation changes the set of included
  (pixel, Gaussian) pairs;
* with the MLP, its gradient equals finite differences of the unrounded FP64
  forward (BF16 rounding is passed straight through, see grad.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import grad as og
from paper_2603_11531_gb300 import synth


def _setup(n=250, seed=5, W=48, H=40, mlp=False):
    s = synth.uniform_scene(n, seed=seed, precision="fp32")
    a = s.attrs.astype(np.float64)
    if mlp:
        s.mlp = synth.random_mlp(seed + 1)
    cam = synth.look_at((0.2, -0.1, -2.6), (0, 0, 0), W, H, 60.0)
    rng = np.random.default_rng(seed)
    dL = rng.normal(size=(H, W, 3))
    return s, a, cam, dL


def _loss_c(a, cam, dL, bg):
    out = oracle.render(a, cam, bg=bg)
    return float((out["rgb"] * dL).sum()), out


def _pairs(a, cam):
    st = og.discrete_structure(a, cam)
    return st["pix"].numpy(), st["gid"].numpy()


def test_restatement_matches_c_oracle():
    s, a, cam, _ = _setup(mlp=True)
    for use_mlp in (False, True):
        ref = oracle.render(a, cam, mlp=s.mlp, use_mlp=use_mlp, rgb_residual=use_mlp, bg=(0.2, 0.1, 0.0))
        st = og.discrete_structure(a, cam, s.mlp, use_mlp, use_mlp)
        p = og.params_from_scene(a, s.mlp)
        img = og.render(p, cam, st, use_mlp=use_mlp, rgb_residual=use_mlp, bg=(0.2, 0.1, 0.0))
        np.testing.assert_allclose(img.detach().numpy(), ref["rgb"], atol=1e-13)


COLS = {"mu": (0, 3), "s": (3, 6), "q": (6, 10), "o": (10, 11), "Y": (11, 23)}


def test_gradient_matches_finite_differences_plain():
    s, a, cam, dL = _setup()
    bg = (0.3, 0.2, 0.1)
    st = og.discrete_structure(a, cam)
    p = og.params_from_scene(a)
    g = og.loss_grad(p, cam, st, dL, bg=bg)
    pix0, gid0 = st["pix"].numpy(), st["gid"].numpy()
    rng = np.random.default_rng(0)
    visible = np.unique(gid0)
    checked = {k: 0 for k in COLS}
    for name, (c0, c1) in COLS.items():
        for _ in range(12):
            i = int(rng.choice(visible))
            col = int(rng.integers(c0, c1))
            h = 1e-6 * max(abs(a[i, col]), 1e-2)
            ap, am = a.copy(), a.copy()
            ap[i, col] += h
            am[i, col] -= h
            pp, pm = _pairs(ap, cam), _pairs(am, cam)
            if not (np.array_equal(pp[0], pix0) and np.array_equal(pp[1], gid0)
                    and np.array_equal(pm[0], pix0) and np.array_equal(pm[1], gid0)):
                continue
            fd = (_loss_c(ap, cam, dL, bg)[0] - _loss_c(am, cam, dL, bg)[0]) / (2 * h)
            ad = g[name].numpy().reshape(len(a), -1)[i, col - c0]
            assert ad == pytest.approx(fd, rel=2e-5, abs=1e-7), (name, i, col, ad, fd)
            checked[name] += 1
    assert all(v >= 6 for v in checked.values()), checked


def test_gradient_matches_finite_differences_mlp_unrounded():
    s, a, cam, dL = _setup(n=150, mlp=True)
    st = og.discrete_structure(a, cam, s.mlp, True, True)
    p = og.params_from_scene(a, s.mlp)
    kw = dict(use_mlp=True, rgb_residual=True, bg=(0.1, 0.1, 0.1), round_bf16=False)
    g = og.loss_grad(p, cam, st, dL, **kw)
    dLt = torch.from_numpy(dL)
    rng = np.random.default_rng(1)

    def L():
        with torch.no_grad():
            return float((og.render(p, cam, st, **kw) * dLt).sum())

    for name in ("w1", "b1", "w2", "b2", "w3", "b3", "mu", "s", "q", "Y"):
        flat = p[name].data.view(-1)
        gf = g[name].view(-1)
        for _ in range(6):
            k = int(rng.integers(0, flat.numel()))
            x0 = float(flat[k])
            h = 1e-6 * max(abs(x0), 1e-2)
            flat[k] = x0 + h
            lp = L()
            flat[k] = x0 - h
            lm = L()
            flat[k] = x0
            fd = (lp - lm) / (2 * h)
            assert float(gf[k]) == pytest.approx(fd, rel=2e-5, abs=1e-7), (name, k)
