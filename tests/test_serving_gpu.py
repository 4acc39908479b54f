"""Continuous-batching server (mgs_server_*) on the GPU.

* each request's image is the same served in a mix as rendered alone (up to
  FP32 accumulation order), for several scenes and resolutions in flight;
* admission respects the device-memory budget; a request that cannot fit
  even alone is refused with MGS_ERR_OOM;
* a bounded wait returns MGS_ERR_TIMEOUT while work is still in flight;
* a request whose tile lists overflow the estimated capacity is re-run.
"""
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
    scenes = []
    for k, n in enumerate((20000, 50000, 120000)):
        s = synth.unbounded_scene(n, seed=70 + k, precision="fp16")
        s.mlp = synth.random_mlp(700 + k)
        scenes.append((s, r.load_scene(s)))
    yield m, r, scenes
    r.close()


def _requests(scenes, n, seed):
    rng = np.random.default_rng(seed)
    sizes = [(320, 240), (640, 480), (400, 300), (512, 288)]
    out = []
    for _ in range(n):
        k = int(rng.integers(len(scenes)))
        W, H = sizes[int(rng.integers(len(sizes)))]
        out.append((k, synth.random_orbit_camera(rng, W, H)))
    return out


def test_mix_equals_alone(env):
    m, r, scenes = env
    from paper_2603_11531_gb300.serving import Server
    reqs = _requests(scenes, 24, seed=1)
    alone = [r.render(scenes[k][1], cam, use_mlp=True)["rgb"] for k, cam in reqs]
    srv = Server(r.ctx, slots=4, max_batch=4, hbm_budget_bytes=2 << 30)
    try:
        outs, tickets = [], []
        opts = m.render_opts(use_mlp=True)
        for k, cam in reqs:
            o = torch.full((cam.height, cam.width, 3), float("nan"), device="cuda")
            outs.append(o)
            tickets.append(srv.submit(scenes[k][1], cam, opts, o))
        for t in tickets:
            srv.wait(t)
        for o, a in zip(outs, alone):
            assert float((o - a).abs().max()) <= 1e-5
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
        info = [srv.ticket(t) for t in tickets]
        assert all(i["t_submit"] <= i["t_admit"] <= i["t_done"] for i in info)
    finally:
        srv.close()
    # and one served image against the oracle (FP16 attributes + BF16 MLP tolerance)
    k, cam = reqs[0]
    ref = oracle.render(scenes[k][0].attrs, cam, mlp=scenes[k][0].mlp, use_mlp=True)
    assert np.abs(outs[0].cpu().numpy() - ref["rgb"]).max() <= 2e-3


def test_admission_respects_memory_budget(env):
    m, r, scenes = env
    from paper_2603_11531_gb300.serving import Server
    budget = 24 << 20
    srv = Server(r.ctx, slots=4, max_batch=4, hbm_budget_bytes=budget)
    try:
        opts = m.render_opts(use_mlp=True)
        tickets, outs = [], []
        for k, cam in _requests(scenes[:2], 10, seed=2):
            o = torch.empty((cam.height, cam.width, 3), device="cuda")
            outs.append(o)
            tickets.append(srv.submit(scenes[k][1], cam, opts, o))
        for t in tickets:
            srv.wait(t)
            assert srv.stats()["workspace_bytes"] <= budget
        # a request that cannot fit even alone is refused
        big = synth.look_at((0, -1, -8), (0, 0, 0), 1920, 1080, 60.0)
        o = torch.empty((1080, 1920, 3), device="cuda")
        t = srv.submit(scenes[2][1], big, opts, o)
        with pytest.raises(m.MGSError) as e:
            srv.wait(t)
        assert e.value.status == m.MGS_ERR_OOM
    finally:
        srv.close()


def test_bounded_wait_times_out_then_completes(env):
    m, r, scenes = env
    from paper_2603_11531_gb300.serving import Server
    srv = Server(r.ctx, slots=2, max_batch=2, hbm_budget_bytes=4 << 30)
    try:
        cam = synth.look_at((0, -1, -8), (0, 0, 0), 1920, 1080, 60.0)
        opts = m.render_opts(use_mlp=True)
        outs = [torch.empty((1080, 1920, 3), device="cuda") for _ in range(6)]
        tickets = [srv.submit(scenes[2][1], cam, opts, o) for o in outs]
        assert srv.wait(tickets[-1], timeout_ms=0.001, allow_timeout=True) == m.MGS_ERR_TIMEOUT
        for t in tickets:
            assert srv.wait(t, timeout_ms=60000) == m.MGS_OK
    finally:
        srv.close()


def test_overflowing_request_is_rerun(env):
    m, r, _ = env
    from paper_2603_11531_gb300.serving import Server
    # a few hundred Gaussians that each cover the whole 1280x720 image: the
    # pair count far exceeds the server's first estimate (max(48 n, 2^20))
    rng = np.random.default_rng(5)
    n = 600
    a = np.zeros((n, 24), np.float32)
    a[:, 0:3] = rng.uniform(-0.05, 0.05, (n, 3))
    a[:, 3:6] = 1.5
    a[:, 6] = 1.0
    a[:, 10] = 0.5
    a[:, 11:23] = rng.normal(0, 0.3, (n, 12))
    scene = synth.Scene(a)
    h = r.load_scene(scene)
    cam = synth.look_at((0, 0, -6), (0, 0, 0), 1280, 720, 60.0)
    ref = r.render(h, cam)["rgb"]
    srv = Server(r.ctx, slots=2, max_batch=2, hbm_budget_bytes=4 << 30)
    try:
        o = torch.empty((720, 1280, 3), device="cuda")
        t = srv.submit(h, cam, m.render_opts(), o)
        srv.wait(t)
        assert float((o - ref).abs().max()) <= 1e-5
    finally:
        srv.close()
        r.unload_scene(h)


def test_batched_raster_with_fp32_sum_tiles(env):
    """Small views rasterised together by the persistent batched rasteriser,
    one of them with a Gaussian whose Eq. 3 weight (exp(32)) sends its tiles
    to the FP32 sums: every served image equals the view rendered alone."""
    m, r, scenes = env
    from paper_2603_11531_gb300.serving import Server
    base = synth.uniform_scene(3000, seed=71).attrs
    big = np.zeros((1, 24), np.float32)
    big[0, 0:3] = (0.0, 0.0, -2.75)
    big[0, 3:6] = (0.002, 0.002, 8.0)
    big[0, 6] = 1.0
    big[0, 10] = 0.9
    big[0, 11:14] = 1.0
    needle = synth.Scene(np.concatenate([base, big]).astype(np.float16))
    hn = r.load_scene(needle)
    cam_n = synth.look_at((0, 0, -3), (0, 0, 0), 320, 240, 60.0)
    opts = m.render_opts()
    reqs = [(hn, cam_n)] + [(scenes[k][1], cam) for k, cam in _requests(scenes, 5, seed=9)]
    alone = [r.render(h, cam)["rgb"] for h, cam in reqs]
    m.mgs_render(r.ws, hn, cam_n, opts, alone[0])
    assert m.mgs_frame_stats(r.ws)["wide_tiles"] > 0
    srv = Server(r.ctx, slots=6, max_batch=6, hbm_budget_bytes=2 << 30)
    try:
        outs = [torch.full((cam.height, cam.width, 3), float("nan"), device="cuda") for _, cam in reqs]
        tickets = [srv.submit(h, cam, opts, o) for (h, cam), o in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t)
        for o, a in zip(outs, alone):
            assert float((o - a).abs().max()) <= 1e-5
    finally:
        srv.close()
        r.unload_scene(hn)
