"""Tensor-core accumulation of A and B (FP16-attribute scenes) on the GPU.

The tensor-core rasteriser computes alpha, the inclusion test and T in FP32
exactly like the FMA rasteriser and sums a_i w_i c_i and a_i w_i with
mma.sync (FP16 alpha, FP16 high + low weight parts, FP32 accumulation).
Bars:
  * per-pixel inclusion counts and T: identical tests, so counts equal the
    oracle's exactly and T agrees with the FMA path to FP32 rounding (1e-5);
  * colours against the FP64 oracle within the FP16-scene tolerance 2e-3;
  * against the FMA rasteriser (MGS_FLAG_RASTER_FMA) within 5e-4: alpha's
    FP16 rounding perturbs each term of A and B by at most 2^-12 relative,
    which moves the normalised colour A / B by at most 2^-12 times the spread
    of the colours involved (< 2 here);
  * chunk edges: lists shorter than, equal to and longer than one chunk of
    16, empty tiles and a ragged image;
  * weights beyond the FP16 range are scaled by a power of two;
  * a Gaussian whose weight the FP16 sums cannot hold next to the others
    (Eq. 3's exp(s_max / d) is unbounded) sends the tiles that list it to
    the FP32 FMA sums, and every other pixel keeps its tensor-core sums.
"""
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


def _both(R, scene, cam, **kw):
    import paper_2603_11531_gb300 as m
    h = R.load_scene(scene)
    try:
        tc = R.render(h, cam, aux=True, count=True, **kw)
        fma = R.render(h, cam, aux=True, count=True, flags=m.MGS_FLAG_RASTER_FMA, **kw)
    finally:
        R.unload_scene(h)
    cv = lambda o: {k: v.cpu().numpy() for k, v in o.items()}
    return cv(tc), cv(fma)


def _check(tc, fma, ref, tol_ref=2e-3, tol_fma=5e-4):
    np.testing.assert_array_equal(tc["count"], ref["count"])
    np.testing.assert_array_equal(fma["count"], ref["count"])
    assert np.abs(tc["aux"][4] - fma["aux"][4]).max() <= 1e-5
    assert np.abs(tc["rgb"] - ref["rgb"]).max() <= tol_ref
    assert np.abs(tc["rgb"] - fma["rgb"]).max() <= tol_fma
    assert np.isfinite(tc["rgb"]).all()


@pytest.mark.parametrize("use_mlp", [False, True])
def test_tc_matches_oracle_and_fma(R, use_mlp):
    scene = synth.unbounded_scene(30000, seed=61, precision="fp16")
    scene.mlp = synth.random_mlp(62)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 320, 240, 60.0)[5]
    tc, fma = _both(R, scene, cam, use_mlp=use_mlp, bg=(0.1, 0.2, 0.3))
    ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=use_mlp, bg=(0.1, 0.2, 0.3),
                        want_count=True)
    _check(tc, fma, ref)


@pytest.mark.parametrize("n", [1, 7, 16, 17, 40])
def test_tc_chunk_edges_ragged_image(R, n):
    """n large Gaussians near the centre of a 250x131 image: most tiles hold
    n entries (below, at and above one chunk of 16), border tiles none."""
    rng = np.random.default_rng(100 + n)
    a = np.zeros((n, 24), np.float32)
    a[:, 0:2] = rng.uniform(-0.3, 0.3, (n, 2))
    a[:, 2] = rng.uniform(-0.2, 0.2, n)
    a[:, 3:6] = rng.uniform(0.15, 0.35, (n, 3))
    a[:, 6:10] = rng.normal(0, 1, (n, 4))
    a[:, 10] = rng.uniform(0.2, 0.9, n)
    a[:, 11:23] = rng.normal(0, 0.4, (n, 12))
    scene = synth.Scene(a.astype(np.float16))
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 250, 131, 60.0)
    tc, fma = _both(R, scene, cam)
    ref = oracle.render(scene.attrs, cam, want_count=True)
    _check(tc, fma, ref)
    assert (ref["count"] == 0).any()          # some pixels see nothing


def test_tc_weights_beyond_fp16_are_scaled(R):
    """A Gaussian 0.25 in front of the camera with scale 3 has
    w > exp(12) > 2^16: without scaling its FP16 weight would overflow."""
    base = synth.uniform_scene(3000, seed=71).attrs
    big = np.zeros((1, 24), np.float32)
    big[0, 0:3] = (0.0, 0.0, -2.75)
    big[0, 3:6] = 3.0
    big[0, 6] = 1.0
    big[0, 10] = 0.02
    big[0, 11:14] = (np.array([0.9, 0.2, 0.1]) - 0.5) / SH_C0
    scene = synth.Scene(np.concatenate([base, big]).astype(np.float16))
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 96, 64, 60.0)
    g = oracle.preprocess(scene.attrs, cam)
    assert g["weight"][-1] > 2.0 ** 16
    tc, fma = _both(R, scene, cam)
    ref = oracle.render(scene.attrs, cam, want_count=True)
    _check(tc, fma, ref)


def test_tc_culling_is_exact(R):
    import paper_2603_11531_gb300 as m
    scene = synth.unbounded_scene(50000, seed=81, precision="fp16")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 400, 272, 60.0)[2]
    h = R.load_scene(scene)
    try:
        a = R.render(h, cam, aux=True, count=True)
        b = R.render(h, cam, aux=True, count=True, flags=m.MGS_FLAG_NO_CULL)
    finally:
        R.unload_scene(h)
    assert bool((a["count"] == b["count"]).all())
    assert float((a["rgb"] - b["rgb"]).abs().max()) <= 1e-5


@pytest.mark.parametrize("x_off", [0.0, 0.02])
def test_tc_weight_span_beyond_fp16_range(R, x_off):
    """Ordinary Gaussians (w about 3) beside one needle with s_max = 8 at view
    depth 0.25, so w = exp(32) > 2^46: one per-frame FP16 scale cannot hold
    both (the ordinary weights would fall below FP16's smallest subnormal).
    On the optical axis the needle covers about 30 pixels across the corner
    of four tiles; 0.02 off axis it smears into a band across the image.
    Every pixel -- those the needle covers, those of its tiles it does not
    cover, and all others -- stays within the FP16-scene bar of the oracle;
    the depth image (Eq. 5) too."""
    base = synth.uniform_scene(3000, seed=71).attrs
    big = np.zeros((1, 24), np.float32)
    big[0, 0:3] = (x_off, 0.0, -2.75)
    big[0, 3:6] = (0.002, 0.002, 8.0)
    big[0, 6] = 1.0
    big[0, 10] = 0.9
    big[0, 11:14] = (np.array([0.9, 0.2, 0.1]) - 0.5) / SH_C0
    scene = synth.Scene(np.concatenate([base, big]).astype(np.float16))
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 96, 64, 60.0)
    g = oracle.preprocess(scene.attrs, cam)
    assert g["weight"][-1] > 2.0 ** 40 and g["visible"][-1] == 1
    tc, fma = _both(R, scene, cam, bg=(0.1, 0.2, 0.3))
    ref = oracle.render(scene.attrs, cam, bg=(0.1, 0.2, 0.3), want_count=True)
    covered = np.array([[oracle.includes(g[-1], x, y) for x in range(96)] for y in range(64)])
    assert covered.any() and (~covered).any()
    _check(tc, fma, ref)
    h = R.load_scene(scene)
    try:
        d = R.render_depth(h, cam)["depth"].cpu().numpy()
    finally:
        R.unload_scene(h)
    dref = oracle.render_depth(scene.attrs, cam)["depth"]
    assert np.abs(d - dref).max() <= 2e-3 * dref.max()
