"""Pins of the sorted comparator in the oracle (App. B, Eq. 11) -- CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth

SH_C0 = 0.5 / math.sqrt(math.pi)


def _rec(mu, s, o, col):
    r = np.zeros(24)
    r[0:3], r[3:6], r[6], r[10] = mu, s, 1.0, o
    r[11:14] = (np.asarray(col, np.float64) - 0.5) / SH_C0
    return r


class Cam:
    def __init__(self, W=32, H=32, f=60.0):
        self.R = np.eye(3, dtype=np.float32)
        self.t = np.zeros(3, np.float32)
        self.fx = self.fy = f
        self.cx, self.cy = W / 2, H / 2
        self.width, self.height, self.znear = W, H, 0.2


def test_two_gaussians_front_to_back():
    """C = c1 a1 + c2 a2 (1 - a1) + (1 - a1)(1 - a2) c_bg with 1 nearer (Eq. 11),
    whatever the order of the input records."""
    cam = Cam()
    near = _rec([0, 0, 2.0], [0.2] * 3, 0.7, [1.0, 0.0, 0.0])
    far = _rec([0, 0, 3.0], [0.3] * 3, 0.6, [0.0, 0.0, 1.0])
    bg = np.array([0.0, 1.0, 0.0])
    for attrs in (np.stack([near, far]), np.stack([far, near])):
        out = oracle.render_sorted(attrs, cam, bg=bg)
        g = out["gauss"]
        i_near = int(np.argmin(g["depth"]))
        px = py = 16
        al = []
        for i in (i_near, 1 - i_near):
            dx, dy = px + 0.5 - g[i]["mean"][0], py + 0.5 - g[i]["mean"][1]
            A, B, C = g[i]["conic"]
            al.append(min(0.99, g[i]["opacity"] * math.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy))))
        c1, c2 = g[i_near]["rgb"], g[1 - i_near]["rgb"]
        exp = c1 * al[0] + c2 * al[1] * (1 - al[0]) + (1 - al[0]) * (1 - al[1]) * bg
        np.testing.assert_allclose(out["rgb"][py, px], exp, atol=1e-12)


def test_same_colour_agrees_with_sort_free():
    """With one colour for all Gaussians both compositing rules give
    (1 - T) c + T c_bg (as long as no pixel terminates early)."""
    s = synth.uniform_scene(120, seed=3)
    a = s.attrs.astype(np.float64)
    a[:, 11:23] = 0.0
    a[:, 11:14] = (np.array([0.2, 0.6, 0.9]) - 0.5) / SH_C0
    a[:, 10] *= 0.3
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 48, 40, 60.0)
    bg = (0.5, 0.1, 0.1)
    srt = oracle.render_sorted(a, cam, bg=bg)
    free = oracle.render(a, cam, bg=bg)
    np.testing.assert_allclose(srt["rgb"], free["rgb"], atol=1e-12)


def test_early_termination_after_opaque_layers():
    """Stacked opaque layers: blending stops before T would fall below 1e-4."""
    cam = Cam()
    recs = [_rec([0, 0, 2.0 + 0.1 * k], [0.3] * 3, 1.0, [k / 10.0, 0.5, 0.5]) for k in range(6)]
    out = oracle.render_sorted(np.stack(recs), cam, want_count=True)
    # centre pixel: a ~ 0.99 per layer -> T = 0.01 after one, 1e-4 after two
    c = out["count"][16, 16]
    assert 1 <= c <= 2
    g = out["gauss"]
    assert c < int((g["visible"] == 1).sum())


@pytest.mark.parametrize("W,H,n,seed", [(32, 32, 60, 0), (37, 21, 40, 1)])
def test_bruteforce_sorted(W, H, n, seed):
    attrs = synth.uniform_scene(n, seed=seed + 200).attrs
    cam = synth.look_at((0.1, 0.2, -2.5), (0, 0, 0), W, H, 60.0)
    bg = np.array([0.05, 0.1, 0.2])
    out = oracle.render_sorted(attrs, cam, bg=bg, want_count=True)
    g = out["gauss"]
    for py in range(H):
        for px in range(W):
            i, j = px // 16, py // 16
            inc = [k for k in range(n) if g[k]["visible"] and g[k]["rect"][0] <= i < g[k]["rect"][2]
                   and g[k]["rect"][1] <= j < g[k]["rect"][3] and oracle.includes(g[k], px, py)]
            inc.sort(key=lambda k: (g[k]["tz32"], k))
            C, T, cnt = np.zeros(3), 1.0, 0
            for k in inc:
                dx, dy = px + 0.5 - g[k]["mean"][0], py + 0.5 - g[k]["mean"][1]
                A, B, Cc = g[k]["conic"]
                al = min(0.99, g[k]["opacity"] * math.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + Cc * dy * dy)))
                if T * (1 - al) < 1e-4:
                    break
                C += g[k]["rgb"] * al * T
                T *= 1 - al
                cnt += 1
            np.testing.assert_allclose(out["rgb"][py, px], C + T * bg, atol=1e-12)
            assert out["count"][py, px] == cnt
