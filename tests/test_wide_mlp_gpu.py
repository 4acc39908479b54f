"""The paper-width enhancement MLP (App. C: MLP_f with 256, 128, 64 neurons,
then the phi / o heads of Eq. 4) on tcgen05, against the FP64 oracle.

Both sides round every layer input to BF16; the GPU accumulates in FP32 on
the tensor cores, so images agree within the FP16/BF16 tolerance (2e-3) and
per-pixel inclusion counts exactly (they do not depend on the MLP)."""
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


@pytest.mark.parametrize("n,prec,res,W,H", [(4096, "fp32", False, 128, 96),
                                             (20000, "fp16", True, 240, 176),
                                             (60000, "fp16", False, 200, 150)])
def test_paper_width_mlp_matches_oracle(R, n, prec, res, W, H):
    scene = synth.unbounded_scene(n, seed=110 + n % 13, precision=prec)
    scene.mlp = synth.random_mlp_paper(111)
    cam = synth.orbit_cameras(8, 8.0, 1.0, W, H, 60.0)[n % 8]
    h = R.load_scene(scene)
    try:
        out = R.render(h, cam, use_mlp=True, rgb_residual=res, count=True)
    finally:
        R.unload_scene(h)
    ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=True, rgb_residual=res,
                        want_count=True)
    np.testing.assert_array_equal(out["count"].cpu().numpy(), ref["count"])
    assert np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max() <= 2e-3


@pytest.mark.parametrize("hidden", [(48, 80, 16), (16, 112, 48)])
def test_uneven_widths_match_oracle(R, hidden):
    """Widths with an odd number of 16-column units: the two warp halves that
    read each layer back split its columns unevenly (one half has none at
    width 16); 5,003 Gaussians leave the last 256-row step ragged."""
    scene = synth.unbounded_scene(5003, seed=121, precision="fp16")
    scene.mlp = synth.random_mlp(122, hidden=hidden)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 144, 96, 60.0)[3]
    h = R.load_scene(scene)
    try:
        out = R.render(h, cam, use_mlp=True, rgb_residual=True, count=True)
    finally:
        R.unload_scene(h)
    ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=True, rgb_residual=True,
                        want_count=True)
    np.testing.assert_array_equal(out["count"].cpu().numpy(), ref["count"])
    assert np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max() <= 2e-3


def test_paper_width_mlp_differs_from_small_mlp(R):
    """Sanity: the three-layer MLP is actually used (different image)."""
    scene = synth.unbounded_scene(8000, seed=5, precision="fp16")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 160, 120, 60.0)[0]
    outs = []
    for mlp in (synth.random_mlp(7), synth.random_mlp_paper(7)):
        scene.mlp = mlp
        h = R.load_scene(scene)
        try:
            outs.append(R.render(h, cam, use_mlp=True)["rgb"].cpu().numpy())
        finally:
            R.unload_scene(h)
    assert np.abs(outs[0] - outs[1]).max() > 1e-2


def test_paper_width_mlp_rejections(R):
    import paper_2603_11531_gb300 as m
    scene = synth.unbounded_scene(1000, seed=6, precision="fp16")
    scene.mlp = synth.random_mlp_paper(8)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 64, 48, 60.0)[0]
    h = R.load_scene(scene)
    try:
        with pytest.raises(m.MGSError) as e:
            R.render(h, cam, use_mlp=True, flags=m.MGS_FLAG_MLP_MMA_SYNC)
        assert e.value.status == m.MGS_ERR_INVALID_ARG
    finally:
        R.unload_scene(h)
    bad = synth.random_mlp(9, hidden=(200, 128, 64))
    with pytest.raises(m.MGSError) as e:
        R.load_scene(scene.attrs, bad)
    assert e.value.status == m.MGS_ERR_INVALID_ARG
