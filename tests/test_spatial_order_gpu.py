"""Scenes stored in spatial (Morton) order (MGS_ORDER_SPATIAL) give the same
results, in the caller's indices, as scenes stored as given: images within
FP32 accumulation-order rounding (1e-5), inclusion counts exact, tile lists
equal as sets to the oracle's, per-Gaussian gradients within 1e-5 relative
of the largest gradient, and the sorted comparator (depth ties broken by the
caller's index) exact in counts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield m, r
    r.close()


def _render(m, r, scene, cam, order, **kw):
    h = r.load_scene(scene, order=order)
    try:
        out = r.render(h, cam, count=True, **kw)
        lists = r.tile_lists()
    finally:
        r.unload_scene(h)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}, lists


@pytest.mark.parametrize("prec,use_mlp,flags", [("fp32", False, 0), ("fp16", True, 0), ("fp32", False, 2)])
def test_spatial_order_same_results(env, prec, use_mlp, flags):
    m, r = env
    scene = synth.unbounded_scene(20000, seed=121, precision=prec)
    scene.mlp = synth.random_mlp(122)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 320, 208, 60.0)[4]
    a, la = _render(m, r, scene, cam, m.MGS_ORDER_AS_GIVEN, use_mlp=use_mlp, flags=flags)
    b, lb = _render(m, r, scene, cam, m.MGS_ORDER_SPATIAL, use_mlp=use_mlp, flags=flags)
    assert np.abs(a["rgb"] - b["rgb"]).max() <= 1e-5
    np.testing.assert_array_equal(a["count"], b["count"])
    np.testing.assert_array_equal(la[0], lb[0])
    for t in range(len(la[0]) - 1):
        assert sorted(la[1][la[0][t]:la[0][t + 1]]) == sorted(lb[1][lb[0][t]:lb[0][t + 1]])
    if not flags:   # and both equal the oracle's lists
        ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=use_mlp)
        np.testing.assert_array_equal(lb[0], ref["offsets"])
        for t in range(len(ref["offsets"]) - 1):
            assert sorted(lb[1][lb[0][t]:lb[0][t + 1]]) == sorted(ref["gids"][ref["offsets"][t]:ref["offsets"][t + 1]])


def test_spatial_order_gradients_in_caller_order(env):
    m, r = env
    scene = synth.unbounded_scene(15000, seed=123, precision="fp32")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 256, 176, 60.0)[6]
    dL = torch.from_numpy(np.random.default_rng(7).normal(size=(176, 256, 3)).astype(np.float32)).cuda()
    grads = []
    for order in (m.MGS_ORDER_AS_GIVEN, m.MGS_ORDER_SPATIAL):
        h = r.load_scene(scene, order=order)
        try:
            rgb = torch.empty((176, 256, 3), device="cuda")
            aux = torch.empty((5, 176, 256), device="cuda")
            opts = m.render_opts()
            m.mgs_render_checked(r.ws, h, cam, opts, rgb, aux, None)
            d = torch.zeros((scene.n, 24), device="cuda")
            m.mgs_render_backward(r.ws, h, cam, opts, dL, aux, d, None)
            torch.cuda.synchronize()
            grads.append(d.cpu().numpy())
        finally:
            r.unload_scene(h)
    scale = np.abs(grads[0]).max()
    assert scale > 0
    assert np.abs(grads[0] - grads[1]).max() <= 1e-5 * scale
