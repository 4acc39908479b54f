"""The allocation-free entry point (mgs_render_static) against mgs_render.

mgs_render_static exists for callers that cannot call cudaMalloc at render
time (code where the device allocator is forbidden or unavailable, or a
real-time loop that must not take the allocator's locks or risk an
out-of-memory failure): its scratch is a fixed __device__ array inside the
library.  Each call here goes through the C-ABI and is compared with the
regular entry point's image on the same inputs, within the FP32 pixel
tolerance the parity tests use; two calls in a row on different inputs check
that the shared array's leftover contents from one call do not leak into the
next.  This file is collected last so that a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest

from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _regular(m, scene, cam, bg):
    r = m.Renderer(0)
    try:
        h = r.load_scene(scene)
        return r.render(h, cam, bg=bg)["rgb"]
    finally:
        r.close()


def test_static_entry_point_matches_regular_render(torch_cuda):
    import paper_2603_11531_gb300 as m
    torch = torch_cuda
    cases = [
        (synth.uniform_scene(4096, seed=1, precision="fp32"),
         synth.look_at((0, 0, -3), (0, 0, 0), 256, 256, 60.0), (0.0, 0.0, 0.0)),
        (synth.unbounded_scene(30000, seed=31, precision="fp16"),
         synth.orbit_cameras(8, 8.0, 1.0, 333, 197, 60.0)[3], (0.2, 0.4, 0.1)),
    ]
    for scene, cam, bg in cases:          # two calls in a row, different inputs
        attrs = torch.from_numpy(scene.attrs).cuda()
        out = torch.full((cam.height, cam.width, 3), float("nan"), device="cuda")
        m.mgs_render_static(attrs, cam, m.render_opts(bg=bg), out)
        ref = _regular(m, scene, cam, bg)
        err = float((out - ref).abs().max())
        assert np.isfinite(err) and err <= TOL_FP32, err


def test_static_entry_point_rejects_sizes_beyond_its_limit(torch_cuda):
    import paper_2603_11531_gb300 as m
    torch = torch_cuda
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 64, 64, 60.0)
    out = torch.empty((64, 64, 3), device="cuda")
    too_many = torch.zeros((131073, 24), dtype=torch.float32, device="cuda")
    with pytest.raises(m.MGSError) as e:
        m.mgs_render_static(too_many, cam, m.render_opts(), out)
    assert e.value.status == m.MGS_ERR_INVALID_ARG
    big = synth.look_at((0, 0, -3), (0, 0, 0), 3840, 2160, 60.0)
    small = torch.zeros((16, 24), dtype=torch.float32, device="cuda")
    with pytest.raises(m.MGSError) as e:
        m.mgs_render_static(small, big, m.render_opts(), out)
    assert e.value.status == m.MGS_ERR_INVALID_ARG
