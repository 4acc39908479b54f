"""Edge cases against the oracle: the largest image extents the C-ABI accepts
(16384 pixels wide or high, 1024 tiles in a row or column), and degenerate
Gaussians (zero scale, zero opacity, a zero quaternion, depth at the near
plane, huge scale), for the FP32 path and the FP16 tensor-core path.
Inclusion counts exact; colours within 1e-4 (FP32) / 2e-3 (FP16)."""
import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu
SH_C0 = 0.28209479177387814


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield r
    r.close()


def _check(R, attrs, cam, tol, bg=(0.1, 0.2, 0.3)):
    h = R.load_scene(attrs)
    try:
        out = R.render(h, cam, count=True, bg=bg)
    finally:
        R.unload_scene(h)
    ref = oracle.render(attrs, cam, bg=bg, want_count=True)
    np.testing.assert_array_equal(out["count"].cpu().numpy(), ref["count"])
    assert np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max() <= tol
    return ref


class StripCam:
    """Pinhole camera at the origin looking down +z with a strip image."""

    def __init__(self, W, H, f=400.0):
        self.R = np.eye(3, dtype=np.float32)
        self.t = np.zeros(3, np.float32)
        self.fx = self.fy = f
        self.cx, self.cy = W / 2, H / 2
        self.width, self.height, self.znear = W, H, 0.2


@pytest.mark.parametrize("W,H", [(16384, 16), (16, 16384)])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_largest_image_extent(R, W, H, prec):
    rng = np.random.default_rng(W + H)
    n = 3000
    a = np.zeros((n, 24), np.float32)
    along = rng.uniform(-18.0, 18.0, n)            # spread over the long axis at depth 1
    a[:, 0] = along if W > H else rng.uniform(-0.01, 0.01, n)
    a[:, 1] = along if H > W else rng.uniform(-0.01, 0.01, n)
    a[:, 2] = 1.0
    a[:, 3:6] = rng.uniform(0.002, 0.02, (n, 3))
    a[:, 6:10] = rng.normal(size=(n, 4))
    a[:, 10] = rng.uniform(0.1, 0.95, n)
    a[:, 11:23] = rng.normal(0, 0.4, (n, 12))
    attrs = a.astype(np.float16) if prec == "fp16" else a
    ref = _check(R, attrs, StripCam(W, H), 2e-3 if prec == "fp16" else 1e-4)
    assert (ref["count"] > 0).sum() > 1000


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_degenerate_gaussians(R, prec):
    rng = np.random.default_rng(5)
    rows = []

    def g(mu, s, q=(1, 0, 0, 0), o=0.7):
        r = np.zeros(24)
        r[0:3], r[3:6], r[6:10], r[10] = mu, s, q, o
        r[11:23] = rng.normal(0, 0.4, 12)
        rows.append(r)

    g([0.0, 0.0, 2.0], [0.0, 0.0, 0.0])                 # zero scale: the 0.3 px dilation only
    g([0.1, 0.0, 2.0], [0.05, 0.05, 0.05], o=0.0)       # zero opacity
    g([-0.1, 0.0, 2.0], [0.05, 0.05, 0.05], q=(0, 0, 0, 0))   # zero quaternion
    g([0.0, 0.1, 0.2], [0.01, 0.01, 0.01])              # at the near plane (culled)
    g([0.0, -0.1, 0.2001], [0.01, 0.01, 0.01])          # just beyond it
    g([0.0, 0.0, 3.0], [50.0, 0.01, 0.01])              # huge, needle-shaped
    g([0.0, 0.0, -1.0], [0.1, 0.1, 0.1])                # behind the camera
    g([0.2, 0.2, 2.5], [0.2, 0.05, 0.1], q=(0.3, 0.9, -0.2, 0.1), o=1.0)   # opacity 1 (clamp)
    attrs = np.stack(rows).astype(np.float16 if prec == "fp16" else np.float32)
    _check(R, attrs, StripCam(96, 80, 100.0), 2e-3 if prec == "fp16" else 1e-4)
