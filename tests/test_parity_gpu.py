"""GPU parity: the CUDA renderer (through the C-ABI) against the FP64 oracle.

Bars (element by element, same seeded inputs):
  * tile lists: equal as sets for every tile (bit-exact integers);
  * per-pixel inclusion counts: equal (the FP32 contract predicate);
  * pixels: max-abs <= 1e-4 (FP32 attributes, plain) and <= 2e-3 (FP16
    attributes and/or the BF16 MLP).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_FP16_MLP = 2e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def R(torch_cuda):
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield r
    r.close()


def _sorted_lists(offsets, gids):
    offsets = np.asarray(offsets, np.int64)
    T = len(offsets) - 1
    tile = np.repeat(np.arange(T), np.diff(offsets))
    g = np.asarray(gids, np.int64)
    order = np.lexsort((g, tile))
    return tile[order], g[order]


def _check_lists(R, ref):
    off, gids = R.tile_lists()
    np.testing.assert_array_equal(off, ref["offsets"])
    t1, g1 = _sorted_lists(off, gids)
    t2, g2 = _sorted_lists(ref["offsets"], ref["gids"])
    np.testing.assert_array_equal(t1, t2)
    np.testing.assert_array_equal(g1, g2)


def _render_both(R, scene, cam, use_mlp=False, residual=False, bg=(0.0, 0.0, 0.0), flags=0):
    h = R.load_scene(scene)
    try:
        out = R.render(h, cam, use_mlp=use_mlp, rgb_residual=residual, bg=bg, aux=True,
                       count=True, flags=flags)
        ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=use_mlp,
                            rgb_residual=residual, bg=bg, want_aux=True, want_count=True)
        _check_lists(R, ref)
    finally:
        R.unload_scene(h)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}, ref


def test_small_fp32_plain_parity(R):
    """4,096 Gaussians, FP32, 256x256: exact tile sets and counts, 1e-4 pixels."""
    scene, cams = synth.workload_small_fp32()
    out, ref = _render_both(R, scene, cams[0])
    np.testing.assert_array_equal(out["count"], ref["count"])
    err = np.abs(out["rgb"] - ref["rgb"]).max()
    assert err <= TOL_FP32, err
    # T and the normalised colour A/B agree too
    np.testing.assert_allclose(out["aux"][4], ref["aux"][4], atol=TOL_FP32)


def test_background_and_ragged_image(R):
    """Non-black c_bg, image size not a multiple of the tile (ragged tail)."""
    scene = synth.uniform_scene(3000, seed=21, precision="fp32")
    cam = synth.look_at((0.4, -0.3, -2.7), (0, 0, 0), 203, 141, 55.0)
    out, ref = _render_both(R, scene, cam, bg=(0.2, 0.7, 0.1))
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP32


def test_culling_is_exact(R, torch_cuda):
    """The per-warp culling only removes Gaussians that include no pixel of
    the block: with and without it every pixel includes exactly the same
    Gaussians (integer counts equal), and the image differs only by the FP32
    rounding of a different accumulation order (tile lists are filled by
    atomics, so their order varies between renders)."""
    import paper_2603_11531_gb300 as m
    scene = synth.unbounded_scene(40000, seed=22, precision="fp16")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 480, 320, 60.0)[2]
    h = R.load_scene(scene)
    try:
        a = R.render(h, cam, aux=True, count=True)
        b = R.render(h, cam, aux=True, count=True, flags=m.MGS_FLAG_NO_CULL)
        assert torch_cuda.equal(a["count"], b["count"])
        assert int(a["count"].sum()) > 0
        assert float((a["rgb"] - b["rgb"]).abs().max()) <= 1e-5
        T_a, T_b = a["aux"][4], b["aux"][4]
        assert float((T_a - T_b).abs().max()) <= 1e-5
    finally:
        R.unload_scene(h)


def test_mlp_fp32_parity(R):
    scene = synth.uniform_scene(4096, seed=1, precision="fp32")
    scene.mlp = synth.random_mlp(11)
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 256, 256, 60.0)
    out, ref = _render_both(R, scene, cam, use_mlp=True, bg=(0.1, 0.1, 0.1))
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP16_MLP


def test_mlp_residual_fp16_parity(R):
    scene = synth.unbounded_scene(20000, seed=23, precision="fp16")
    scene.mlp = synth.random_mlp(12)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 320, 212, 60.0)[5]
    out, ref = _render_both(R, scene, cam, use_mlp=True, residual=True)
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP16_MLP


def test_edge_cases(R, torch_cuda):
    torch = torch_cuda
    # one Gaussian; tiny image of one pixel; one Gaussian behind the camera
    one = synth.uniform_scene(1, seed=3, precision="fp32")
    for cam in (synth.look_at((0, 0, -3), (0, 0, 0), 1, 1, 60.0),
                synth.look_at((0, 0, -3), (0, 0, 0), 17, 33, 60.0),
                synth.look_at((0, 0, -3), (0, 0, -6), 32, 32, 60.0)):
        out, ref = _render_both(R, one, cam, bg=(0.3, 0.2, 0.1))
        np.testing.assert_array_equal(out["count"], ref["count"])
        assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP32
    # empty scene: background everywhere
    empty = synth.Scene(np.zeros((0, 24), np.float32))
    h = R.load_scene(empty)
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 40, 24, 60.0)
    out = R.render(h, cam, bg=(0.25, 0.5, 0.75), count=True)
    R.unload_scene(h)
    exp = torch.tensor([0.25, 0.5, 0.75], device="cuda").expand(24, 40, 3)
    assert torch.equal(out["rgb"], exp)
    assert int(out["count"].sum()) == 0


def test_errors_are_reported(R, torch_cuda):
    import paper_2603_11531_gb300 as m
    scene = synth.uniform_scene(16, seed=4, precision="fp32")
    h = R.load_scene(scene)
    try:
        cam = synth.look_at((0, 0, -3), (0, 0, 0), 32, 32, 60.0)
        with pytest.raises(m.MGSError) as e:
            R.render(h, cam, use_mlp=True)
        assert e.value.status == m.MGS_ERR_INVALID_ARG
        bad = synth.look_at((0, 0, -3), (0, 0, 0), 32, 32, 60.0)
        bad.width = 0
        with pytest.raises(m.MGSError) as e:
            R.render(h, bad)
        assert e.value.status == m.MGS_ERR_INVALID_ARG
    finally:
        R.unload_scene(h)


def test_overflow_is_detected_and_recovered(torch_cuda):
    """A workspace too small for the tile lists reports MGS_ERR_OVERFLOW at
    sync; the checked render grows it and matches a fresh render."""
    import paper_2603_11531_gb300 as m
    torch = torch_cuda
    scene = synth.uniform_scene(4096, seed=1, precision="fp32")
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 256, 256, 60.0)
    r = m.Renderer(0)
    try:
        h = r.load_scene(scene)
        m.mgs_workspace_reserve(r.ws, scene.n, 256, 256, 1000)
        # the default render sizes from the scene only if nothing is reserved
        rgb = torch.empty((256, 256, 3), device="cuda")
        m.mgs_render(r.ws, h, cam, m.render_opts(), rgb)
        st, pairs = m.mgs_workspace_sync(r.ws, allow_overflow=True)
        assert st == m.MGS_ERR_OVERFLOW and pairs > 1000
        out = r.render(h, cam)   # checked: succeeds now
        ref = oracle.render(scene.attrs, cam)
        assert np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max() <= TOL_FP32
    finally:
        r.close()


def test_render_to_host_matches_device(R, torch_cuda):
    import paper_2603_11531_gb300 as m
    torch = torch_cuda
    scene = synth.uniform_scene(2000, seed=5, precision="fp16")
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 96, 80, 60.0)
    h = R.load_scene(scene)
    try:
        dev = R.render(h, cam)["rgb"]
        host = torch.empty((80, 96, 3), dtype=torch.float32).pin_memory()
        m.mgs_render_to_host(R.ws, h, cam, m.render_opts(), host)
        torch.cuda.synchronize()
        # same Gaussians per pixel; list order (hence FP32 rounding) may differ
        assert float((host - dev.cpu()).abs().max()) <= 1e-5
    finally:
        R.unload_scene(h)


@pytest.mark.slow
def test_unbounded_600k_full_size_sampled(R, error_report):
    """The benchmark workload (600k FP16 Gaussians, BF16 MLP, 1600x1063):
    all tile lists exact; counts and pixels on a sample of tiles."""
    scene, cams = synth.workload_unbounded_600k(n_poses=64)
    errs = []
    for pose in (0, 21):
        cam = cams[pose]
        h = R.load_scene(scene)
        try:
            out = R.render(h, cam, use_mlp=True, aux=False, count=True)
            g = oracle.preprocess(scene.attrs, cam, scene.mlp, use_mlp=True)
            off, gids = oracle.bin_tiles(g, cam.width, cam.height)
            _check_lists(R, {"offsets": off, "gids": gids})
            tx, ty = oracle.tiles(cam.width, cam.height)
            rng = np.random.default_rng(pose)
            # the heaviest tiles plus a random sample, and the ragged last row
            heavy = np.argsort(np.diff(off))[-6:]
            sample = np.unique(np.concatenate([heavy, rng.integers(0, tx * ty, 24),
                                               np.arange((ty - 1) * tx, (ty - 1) * tx + 4)]))
            rgb = out["rgb"].cpu().numpy()
            cnt = out["count"].cpu().numpy()
            for t in sample:
                ref_rgb, _, ref_cnt = oracle.rasterize(g, off, gids, cam.width, cam.height,
                                                       tile_range=(int(t), int(t) + 1),
                                                       want_count=True)
                x0, y0 = (t % tx) * 16, (t // tx) * 16
                sl = (slice(y0, min(y0 + 16, cam.height)), slice(x0, min(x0 + 16, cam.width)))
                np.testing.assert_array_equal(cnt[sl], ref_cnt[sl])
                e = np.abs(rgb[sl] - ref_rgb[sl])
                assert e.max() <= TOL_FP16_MLP, (t, e.max())
                errs.append(e.ravel())
        finally:
            R.unload_scene(h)
    flat = np.concatenate(errs)
    error_report["unbounded_600k_1600x1063_fp16_mlp"] = {
        "poses": [0, 21], "tiles_per_pose": "heaviest 6 + 24 random + 4 of the ragged last row",
        "max_abs": float(flat.max()), "mean_abs": float(flat.mean())}


def test_repeat_renders_agree(R, torch_cuda):
    """Tile-list order may differ between runs (atomic scatter); the image
    may differ only by FP32 rounding."""
    scene = synth.unbounded_scene(100000, seed=24, precision="fp16")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 640, 480, 60.0)[1]
    h = R.load_scene(scene)
    try:
        a = R.render(h, cam)["rgb"]
        b = R.render(h, cam)["rgb"]
        assert float((a - b).abs().max()) <= 1e-5
    finally:
        R.unload_scene(h)


def test_all_poses_reduced_resolution(R):
    """Every orbit pose of the benchmark path at 400x266 with 60k Gaussians."""
    scene = synth.unbounded_scene(60000, seed=25, precision="fp16")
    scene.mlp = synth.random_mlp(26)
    h = R.load_scene(scene)
    try:
        for cam in synth.orbit_cameras(16, 8.0, 1.0, 400, 266, 60.0):
            out = R.render(h, cam, use_mlp=True, count=True)
            ref = oracle.render(scene.attrs, cam, mlp=scene.mlp, use_mlp=True, want_count=True)
            np.testing.assert_array_equal(out["count"].cpu().numpy(), ref["count"])
            err = np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max()
            assert err <= TOL_FP16_MLP, err
    finally:
        R.unload_scene(h)
    assert math.isfinite(err)


def test_binning_work_plan_cases(R):
    """Tile lists and pixels for scenes that stress the binning work plan
    (equal shares of the 32-Gaussian groups' pair counts plus a per-group
    visit charge): long runs of groups without pairs between visible ones,
    a ragged last group, fewer plan units than warps, and one Gaussian that
    covers every tile among many small ones."""
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 200, 136, 60.0)
    # 20,011 Gaussians: index ranges [3000, 9000) and [12000, 19000) moved
    # behind the camera, so thousands of consecutive groups have no pairs
    sc = synth.uniform_scene(20011, seed=41, precision="fp32")
    a = sc.attrs.copy()
    a[3000:9000, 2] = -20.0
    a[12000:19000, 2] = -20.0
    out, ref = _render_both(R, synth.Scene(a), cam, bg=(0.1, 0.2, 0.3))
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP32
    # 37 Gaussians (two groups, the second ragged): far fewer plan units than warps
    few = synth.uniform_scene(37, seed=42, precision="fp32")
    out, ref = _render_both(R, few, cam)
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP32
    # one Gaussian at the centre, scaled to cover the whole image, among 5,000
    big = synth.uniform_scene(5000, seed=43, precision="fp32").attrs.copy()
    big[2500, 0:3] = 0.0
    big[2500, 3:6] = 3.0
    out, ref = _render_both(R, synth.Scene(big), cam)
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= TOL_FP32


@pytest.mark.parametrize("prec,use_mlp,tol", [("fp32", False, TOL_FP32), ("fp16", True, TOL_FP16_MLP)])
def test_two_tile_bands(R, prec, use_mlp, tol):
    """4096x2304 has 256 x 144 tiles, more than one shared-memory band of
    the binning (32,768 words: 127 tile rows of 257 difference-array words at
    this width): both bands hold listed pairs (means spread over [-3, 3]^3
    reach the bottom tile rows)."""
    sc = synth.uniform_scene(3000, seed=61, precision=prec)
    a = sc.attrs.copy()
    a[:, 0:3] *= 3.0
    scene = synth.Scene(a)
    scene.mlp = synth.random_mlp(62)
    cam = synth.look_at((0, 0, -10), (0, 0, 0), 4096, 2304, 60.0)
    out, ref = _render_both(R, scene, cam, use_mlp=use_mlp, bg=(0.1, 0.2, 0.3))
    assert int(ref["offsets"][-1] - ref["offsets"][127 * 256]) > 0
    np.testing.assert_array_equal(out["count"], ref["count"])
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= tol


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_row_resolution_anisotropic(R, prec):
    """Binning resolves each rectangle row of a Gaussian from a few
    evaluations of the FP32 tile test (the passing tiles of a row form one
    interval), not one test per tile.  Stress it with needle-thin ellipses
    at every angle (a few pixels wide, hundreds long), Gaussians whose means
    lie far outside the image, image-sized ones and tiny ones, at an odd
    resolution: the lists must equal the oracle's per-tile lists as sets,
    and the per-pixel counts must agree."""
    rng = np.random.default_rng(71)
    n = 3000
    a = synth.uniform_scene(n, seed=72, precision="fp32").attrs.astype(np.float64)
    kind = rng.integers(0, 4, n)
    s = a[:, 3:6]
    # needles: one long axis, two very short ones
    nd = kind == 0
    s[nd, 0] = np.exp(rng.uniform(-1.5, 0.5, nd.sum()))
    s[nd, 1] = np.exp(rng.uniform(-8.0, -5.0, nd.sum()))
    s[nd, 2] = np.exp(rng.uniform(-8.0, -5.0, nd.sum()))
    # flat discs seen at grazing angles
    fl = kind == 1
    s[fl, 0:2] = np.exp(rng.uniform(-2.0, -0.5, (fl.sum(), 2)))
    s[fl, 2] = 1e-4
    # means far outside the frustum's centre, large enough to reach the image
    far = kind == 2
    a[far, 0:2] = rng.uniform(-4.0, 4.0, (far.sum(), 2))
    s[far, :] = np.exp(rng.uniform(-1.0, 0.3, (far.sum(), 3)))
    # tiny ones
    ti = kind == 3
    s[ti, :] = np.exp(rng.uniform(-7.0, -5.0, (ti.sum(), 3)))
    a[:, 3:6] = s
    scene = synth.Scene(a.astype(np.float32 if prec == "fp32" else np.float16))
    cam = synth.look_at((0.3, -0.2, -3.2), (0, 0, 0), 1013, 771, 70.0)
    out, ref = _render_both(R, scene, cam, bg=(0.1, 0.2, 0.3))
    assert int(ref["offsets"][-1]) > 500_000
    np.testing.assert_array_equal(out["count"], ref["count"])
    tol = TOL_FP32 if prec == "fp32" else TOL_FP16_MLP
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= tol
