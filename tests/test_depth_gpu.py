"""Depth image for the Eq. 5 distillation (mgs_render_depth) against the
oracle: D = sum d a w / sum a w with Eq. 2's inclusion test and weights.

Bars: pixels with no included Gaussian are exactly 0 on both sides; FP32
attributes: |D - D_ref| <= 1e-5 x max D (FP32 sums of a few hundred terms);
FP16 attributes + BF16 MLP: <= 2e-3 x max D, the relative weight error the
colour tolerance allows, applied to a depth spread up to max D (the
denominator is the tensor-core sum of FP16 alphas there; with
MGS_FLAG_RASTER_FMA both sums are FP32).  The colour image of the same call
equals mgs_render's with the same options within 1e-5."""
import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield r
    r.close()


def _run(R, scene, cam, use_mlp=False, flags=0):
    h = R.load_scene(scene)
    try:
        out = R.render_depth(h, cam, use_mlp=use_mlp, flags=flags)
        plain = R.render(h, cam, use_mlp=use_mlp, flags=flags)
    finally:
        R.unload_scene(h)
    return out["depth"].cpu().numpy(), out["rgb"].cpu().numpy(), plain["rgb"].cpu().numpy()


def test_depth_fp32_small(R):
    scene, cams = synth.workload_small_fp32()
    cam = cams[0]
    d, rgb, plain = _run(R, scene, cam)
    ref = oracle.render_depth(scene.attrs, cam)["depth"]
    assert ((d == 0) == (ref == 0)).all()
    assert np.abs(d - ref).max() <= 1e-5 * ref.max()
    assert np.abs(rgb - plain).max() <= 1e-5


@pytest.mark.parametrize("fma", [False, True])
def test_depth_fp16_mlp_unbounded(R, fma):
    import paper_2603_11531_gb300 as m
    scene = synth.unbounded_scene(40000, seed=51, precision="fp16")
    scene.mlp = synth.random_mlp(52)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 272, 180, 60.0)[1]
    d, rgb, plain = _run(R, scene, cam, use_mlp=True, flags=m.MGS_FLAG_RASTER_FMA if fma else 0)
    ref = oracle.render_depth(scene.attrs, cam, mlp=scene.mlp, use_mlp=True)["depth"]
    assert ((d == 0) == (ref == 0)).all()
    assert np.abs(d - ref).max() <= 2e-3 * ref.max()
    assert np.abs(rgb - plain).max() <= 1e-5


def test_depth_rejects_sorted(R):
    import paper_2603_11531_gb300 as m
    scene = synth.uniform_scene(100, seed=3)
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 64, 48, 60.0)
    h = R.load_scene(scene)
    try:
        with pytest.raises(m.MGSError) as e:
            R.render_depth(h, cam, flags=m.MGS_FLAG_SORTED)
        assert e.value.status == m.MGS_ERR_INVALID_ARG
    finally:
        R.unload_scene(h)
