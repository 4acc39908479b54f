"""Pins of the oracle's depth image (Sec. 3.2, Eq. 5 reading:
D = sum d a w / sum a w over the included Gaussians) -- CPU only."""
import math

import numpy as np

import oracle
from paper_2603_11531_gb300 import synth

SH_C0 = 0.5 / math.sqrt(math.pi)


class Cam:
    """Camera at the origin looking down +z: view depth = world z."""

    def __init__(self, W=40, H=32, f=50.0):
        self.R = np.eye(3, dtype=np.float32)
        self.t = np.zeros(3, np.float32)
        self.fx = self.fy = f
        self.cx, self.cy = W / 2, H / 2
        self.width, self.height, self.znear = W, H, 0.2


def _rec(mu, s, o, rgb=(0.5, 0.5, 0.5)):
    r = np.zeros(24)
    r[0:3], r[3:6], r[6], r[10] = mu, s, 1.0, o
    r[11:14] = (np.asarray(rgb, np.float64) - 0.5) / SH_C0
    return r


def test_single_gaussian_depth_is_its_depth():
    out = oracle.render_depth(np.stack([_rec([0.0, 0.0, 2.5], [0.2] * 3, 0.8)]), Cam())
    g = out["gauss"]
    ref = oracle.render(np.stack([_rec([0.0, 0.0, 2.5], [0.2] * 3, 0.8)]), Cam(), want_count=True)
    covered = ref["count"] > 0
    assert covered.any() and (~covered).any()
    np.testing.assert_allclose(out["depth"][covered], g["depth"][0], rtol=1e-15)
    assert (out["depth"][~covered] == 0.0).all()
    assert abs(g["depth"][0] - 2.5) < 1e-6


def test_fronto_parallel_plane_has_constant_depth():
    """Gaussians at different (x, y) on the plane z = 3: every covered pixel
    has depth 3 whatever the weights, opacities and overlaps."""
    rng = np.random.default_rng(4)
    recs = [_rec([rng.uniform(-0.8, 0.8), rng.uniform(-0.6, 0.6), 3.0],
                 rng.uniform(0.05, 0.2, 3), rng.uniform(0.1, 0.95)) for _ in range(30)]
    out = oracle.render_depth(np.stack(recs), Cam())
    d = out["depth"]
    assert (d > 0).sum() > 100
    np.testing.assert_allclose(d[d > 0], 3.0, rtol=1e-6)


def test_depth_equals_normalised_colour_carrying_depth():
    """With view-independent colours c_r = d / 10, the colour sum A_r / B of
    Eq. 2 (pinned separately) equals D / 10 at every covered pixel."""
    rng = np.random.default_rng(5)
    recs = []
    for _ in range(40):
        z = rng.uniform(2.0, 6.0)
        recs.append(_rec([rng.uniform(-1, 1), rng.uniform(-0.8, 0.8), z],
                         rng.uniform(0.05, 0.3, 3), rng.uniform(0.1, 0.95), (z / 10.0, 0.3, 0.3)))
    a = np.stack(recs)
    cam = Cam(48, 36, 40.0)
    dep = oracle.render_depth(a, cam)["depth"]
    ref = oracle.render(a, cam, want_aux=True, want_count=True)
    A, B = ref["aux"][0], ref["aux"][3]
    cov = B > 0
    assert cov.sum() > 200
    np.testing.assert_allclose(dep[cov], 10.0 * A[cov] / B[cov], rtol=1e-6)
    assert (dep[~cov] == 0.0).all()


def test_depth_permutation_invariant():
    a = synth.uniform_scene(200, seed=9).attrs.astype(np.float64)
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 50, 38, 60.0)
    d1 = oracle.render_depth(a, cam)["depth"]
    d2 = oracle.render_depth(a[np.random.default_rng(1).permutation(len(a))], cam)["depth"]
    np.testing.assert_allclose(d1, d2, rtol=1e-12, atol=1e-12)
