"""The large workload -- 6M Gaussians of the unbounded distribution, FP16
attributes, BF16 MLP, 3840x2160 -- against the FP64 oracle on sampled tiles,
for the sort-free renderer (Sec. 3.1, Eq. 2-4) and the sorted comparator
(App. B, Eq. 11).  Above 2^21 Gaussians the scene is stored in spatial
(Morton) order and the tile lists hold about 560 M entries; the sampled
tiles' lists must equal the oracle's as sets (caller indices), their
per-pixel inclusion counts exactly (the comparator's blend counts within
one), and their pixels within the FP16-scene bar.

The oracle projects all 6M Gaussians (worker processes, its own routine per
Gaussian); binning and rasterisation of the sampled tiles use the Gaussians
whose 3-sigma rectangle contains one of them, which are all that can be
listed there.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pool
from paper_2603_11531_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 2e-3


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield r
    r.close()


def test_large_6m_4k_sampled_tiles(R, error_report):
    import paper_2603_11531_gb300 as m
    scene, cam = synth.workload_large_6m()
    W, H = cam.width, cam.height
    tx, ty = oracle.tiles(W, H)
    h = R.load_scene(scene)
    try:
        out = R.render(h, cam, use_mlp=True, count=True)
        n_tiles, n_pairs = m.mgs_tile_lists(R.ws)
        off_d = torch.empty(n_tiles + 1, dtype=torch.int32, device="cuda")
        gid_d = torch.empty(n_pairs, dtype=torch.int32, device="cuda")
        m.mgs_tile_lists(R.ws, off_d, gid_d)
        srt = R.render(h, cam, use_mlp=True, count=True, flags=m.MGS_FLAG_SORTED)
    finally:
        R.unload_scene(h)
    assert n_pairs > 4e8
    off_gpu = off_d.cpu().numpy().view(np.uint32).astype(np.int64)
    rgb, cnt = out["rgb"].cpu().numpy(), out["count"].cpu().numpy()
    srgb, scnt = srt["rgb"].cpu().numpy(), srt["count"].cpu().numpy()

    g = oracle_pool.preprocess(scene.attrs, cam, scene.mlp, use_mlp=True)
    rng = np.random.default_rng(5)
    lens = np.diff(off_gpu)
    sample = np.unique(np.concatenate([np.argsort(lens)[-6:], rng.integers(0, tx * ty, 20),
                                       np.arange((ty - 1) * tx, (ty - 1) * tx + 3),
                                       np.arange(tx - 3, tx)]))
    vis = g["visible"] == 1
    rect = g["rect"]
    keep = np.zeros(len(g), bool)
    for t in sample:
        i, j = t % tx, t // tx
        keep |= vis & (rect[:, 0] <= i) & (i < rect[:, 2]) & (rect[:, 1] <= j) & (j < rect[:, 3])
    idx = np.flatnonzero(keep)
    gs = np.ascontiguousarray(g[idx])
    del g
    off_s, gids_s = oracle.bin_tiles(gs, W, H)

    errs, serrs = [], []
    for t in sample:
        t = int(t)
        mine = np.sort(gid_d[off_gpu[t]:off_gpu[t + 1]].cpu().numpy().astype(np.int64))
        ref = np.sort(idx[gids_s[off_s[t]:off_s[t + 1]]])
        np.testing.assert_array_equal(mine, ref)
        x0, y0 = (t % tx) * 16, (t // tx) * 16
        sl = (slice(y0, min(y0 + 16, H)), slice(x0, min(x0 + 16, W)))
        r_rgb, _, r_cnt = oracle.rasterize(gs, off_s, gids_s, W, H, tile_range=(t, t + 1),
                                           want_count=True)
        np.testing.assert_array_equal(cnt[sl], r_cnt[sl])
        e = np.abs(rgb[sl] - r_rgb[sl])
        assert e.max() <= TOL, (t, e.max())
        errs.append(e)
        s_rgb, s_cnt = oracle.rasterize_sorted(gs, off_s, gids_s, W, H, tile_range=(t, t + 1),
                                               want_count=True)
        assert np.abs(scnt[sl] - s_cnt[sl]).max() <= 1
        e = np.abs(srgb[sl] - s_rgb[sl])
        assert e.max() <= TOL, (t, e.max())
        serrs.append(e)
    flat = np.concatenate([e.ravel() for e in errs])
    sflat = np.concatenate([e.ravel() for e in serrs])
    error_report["large_6m_3840x2160_sort_free"] = {
        "tiles": len(sample), "max_abs": float(flat.max()), "mean_abs": float(flat.mean())}
    error_report["large_6m_3840x2160_sorted"] = {
        "tiles": len(sample), "max_abs": float(sflat.max()), "mean_abs": float(sflat.mean())}
