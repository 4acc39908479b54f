"""Error of the GPU path against the FP64 oracle, stated per workload.

Each test checks the parity bar of its workload and records max-abs and
mean-abs errors in the session's error report (written to $MGS_ERROR_REPORT
when set; the 600k, 6M and gradient workloads are recorded by their own
parity tests):

  * small FP32 workload (4,096 Gaussians, 256x256): the whole image;
  * serving: images served by the continuous-batching server for scenes of
    the serving set at the serving resolutions, whole images;
  * the BF16 deployment of the MLP: the GPU image against the oracle with
    the MLP's BF16 input rounding, and against the FP64 MLP without it (the
    latter is a property of running Eq. 4 in BF16, not of the kernels).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import grad as og
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield r
    r.close()


def _stats(a, b):
    e = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return {"max_abs": float(e.max()), "mean_abs": float(e.mean())}


def test_error_small_fp32(R, error_report):
    scene, cams = synth.workload_small_fp32()
    h = R.load_scene(scene)
    try:
        out = R.render(h, cams[0])["rgb"].cpu().numpy()
    finally:
        R.unload_scene(h)
    ref = oracle.render(scene.attrs, cams[0])["rgb"]
    st = _stats(out, ref)
    assert st["max_abs"] <= 1e-4
    error_report["small_4096_256x256_fp32"] = dict(st, pixels="all")


def test_error_served_images(R, error_report):
    """Requests for three scenes of the serving set (50k, 90k, 160k
    Gaussians, FP16, BF16 MLP) at 640x480 and 1280x720, all in flight at
    once through the server; every served image against the oracle."""
    import paper_2603_11531_gb300 as m
    from paper_2603_11531_gb300.serving import Server
    scenes = synth.serving_scenes(synth.SERVING_SIZES[:3])
    rng = np.random.default_rng(12)
    handles = [R.load_scene(s) for s in scenes]
    srv = Server(R.ctx, slots=4, max_batch=4, hbm_budget_bytes=4 << 30)
    try:
        reqs = []
        for k in range(6):
            W, H = synth.SERVING_RESOLUTIONS[k % 2]
            cam = synth.random_orbit_camera(rng, W, H)
            out = torch.empty((H, W, 3), device="cuda")
            reqs.append((k % 3, cam, out, srv.submit(handles[k % 3], cam, m.render_opts(use_mlp=True), out)))
        worst = {"max_abs": 0.0, "mean_abs": 0.0}
        for k, cam, out, t in reqs:
            srv.wait(t)
            sc = scenes[k]
            ref = oracle.render(sc.attrs, cam, mlp=sc.mlp, use_mlp=True)["rgb"]
            st = _stats(out.cpu().numpy(), ref)
            assert st["max_abs"] <= 2e-3, st
            worst = {"max_abs": max(worst["max_abs"], st["max_abs"]),
                     "mean_abs": max(worst["mean_abs"], st["mean_abs"])}
    finally:
        srv.close()
        for hd in handles:
            R.unload_scene(hd)
    error_report["serving_50k_90k_160k_640x480_1280x720"] = dict(worst, requests=6, pixels="all")


def test_error_bf16_mlp_against_unrounded(R, error_report):
    """100k Gaussians of the unbounded distribution with the BF16 MLP at
    400x266: the GPU image against the oracle with and without the BF16
    rounding of the MLP inputs (the FP64 restatement of the oracle)."""
    scene = synth.unbounded_scene(100000, seed=13, precision="fp16")
    scene.mlp = synth.random_mlp(14)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 400, 266, 60.0)[0]
    h = R.load_scene(scene)
    try:
        out = R.render(h, cam, use_mlp=True)["rgb"].cpu().numpy()
    finally:
        R.unload_scene(h)
    ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=True)["rgb"]
    st = og.discrete_structure(scene.attrs, cam, scene.mlp, use_mlp=True)
    p = og.params_from_scene(scene.attrs, scene.mlp)
    with torch.no_grad():
        unrounded = og.render(p, cam, st, use_mlp=True, round_bf16=False).numpy()
    a, b = _stats(out, ref), _stats(out, unrounded)
    assert a["max_abs"] <= 2e-3
    error_report["bf16_mlp_100k_400x266"] = {"vs_oracle_bf16_inputs": a,
                                             "vs_fp64_mlp_unrounded": b}
