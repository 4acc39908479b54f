"""The allocation-free entry point (mgs_render_static) against mgs_render and
the FP64 oracle.

mgs_render_static exists for callers that cannot call cudaMalloc at render
time (code where the device allocator is forbidden or unavailable, or a
real-time loop that must not take the allocator's locks or risk an
out-of-memory failure): its scratch is a fixed __device__ array inside the
library.  Each call here goes through the C-ABI and is compared with the
regular entry point's image and with the oracle's on the same inputs, within
the pixel tolerances the parity tests use.  Calls run in a row on different
inputs -- a small one, a larger one, then a small one again -- so that
leftover records, counts or lists of a larger call in the shared array would
show up in the next, smaller one; a call that needs more (tile, Gaussian)
pairs than the array holds must report MGS_ERR_OVERFLOW and leave the next
call correct.  This file is collected last so that a stop-at-first-failure
run has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_FP16 = 2e-3


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


def _cases():
    small = (synth.uniform_scene(4096, seed=1, precision="fp32"),
             synth.look_at((0, 0, -3), (0, 0, 0), 256, 256, 60.0), (0.0, 0.0, 0.0), TOL_FP32)
    large = (synth.unbounded_scene(30000, seed=31, precision="fp16"),
             synth.orbit_cameras(8, 8.0, 1.0, 333, 197, 60.0)[3], (0.2, 0.4, 0.1), TOL_FP16)
    return small, large


def _static_render(m, torch, scene, cam, bg):
    attrs = torch.from_numpy(scene.attrs).cuda()
    out = torch.full((cam.height, cam.width, 3), float("nan"), device="cuda")
    m.mgs_render_static(attrs, cam, m.render_opts(bg=bg), out)
    return out


def test_static_entry_point_matches_regular_render_and_oracle(torch_cuda):
    import paper_2603_11531_gb300 as m
    torch = torch_cuda
    small, large = _cases()
    for scene, cam, bg, tol in (small, large, small):   # small after large: no leftovers
        out = _static_render(m, torch, scene, cam, bg)
        ref = _regular(m, scene, cam, bg)
        err = float((out - ref).abs().max())
        assert np.isfinite(err) and err <= 1e-5, err        # same arithmetic, list order aside
        orc = oracle.render(scene.attrs, cam, bg=bg)["rgb"]
        err_o = float(np.abs(out.cpu().numpy() - orc).max())
        assert np.isfinite(err_o) and err_o <= tol, err_o


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
    out_big = torch.empty((2160, 3840, 3), device="cuda")
    with pytest.raises(m.MGSError) as e:
        m.mgs_render_static(small, big, m.render_opts(), out_big)
    assert e.value.status == m.MGS_ERR_INVALID_ARG
    # flags the entry point does not honour are refused, not ignored
    for flags in (m.MGS_FLAG_SORTED, m.MGS_FLAG_MLP_MMA_SYNC):
        with pytest.raises(m.MGSError) as e:
            m.mgs_render_static(small, cam, m.render_opts(flags=flags), out)
        assert e.value.status == m.MGS_ERR_INVALID_ARG


def test_static_entry_point_overflow_then_recovers(torch_cuda):
    import paper_2603_11531_gb300 as m
    torch = torch_cuda
    # 12,000 large Gaussians at 640x480 need about 5 M (tile, Gaussian) pairs,
    # more than the 4,194,304 the array holds
    rng = np.random.default_rng(77)
    a = np.zeros((12000, 24), np.float32)
    a[:, 0:3] = rng.uniform(-0.3, 0.3, (12000, 3))
    a[:, 3:6] = 0.4
    a[:, 6] = 1.0
    a[:, 10] = 0.5
    a[:, 11:23] = rng.normal(0.0, 0.3, (12000, 12))
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 640, 480, 60.0)
    out = torch.empty((480, 640, 3), device="cuda")
    with pytest.raises(m.MGSError) as e:
        m.mgs_render_static(torch.from_numpy(a).cuda(), cam, m.render_opts(), out)
    assert e.value.status == m.MGS_ERR_OVERFLOW
    scene, cam2, bg, tol = _cases()[0]
    out2 = _static_render(m, torch, scene, cam2, bg)
    orc = oracle.render(scene.attrs, cam2, bg=bg)["rgb"]
    err = float(np.abs(out2.cpu().numpy() - orc).max())
    assert np.isfinite(err) and err <= tol, err
