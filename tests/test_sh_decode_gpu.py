"""Load-time SH decode (Sec. 3.2, Eq. 6, mgs_decode_sh) against the oracle.

Bars: FP32 attributes: |Y - Y_ref| <= 1e-5 (FP32 accumulation of 70 terms
with |Y| ~ 1); FP16 attributes: |Y - Y_ref| <= 2^-11 |Y_ref| + 1e-5 (half a
binary16 ulp plus the FP32 error); the other 12 attribute columns are not
touched; decoding then rendering agrees with the oracle decoding then
rendering within the FP16 tolerance 2e-3."""
import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as m
    r = m.Renderer(0)
    yield m, r, torch
    r.close()


@pytest.mark.parametrize("prec,n", [("fp32", 20000), ("fp16", 20011), ("fp16", 1)])
def test_decode_matches_oracle(env, prec, n):
    m, r, torch = env
    md, mv = synth.random_sh_decoders(30 + n % 7)
    h = synth.compressed_sh_features(n, seed=31, precision=prec)
    dt = torch.float16 if prec == "fp16" else torch.float32
    attrs = torch.full((n, 24), 7.0, dtype=dt, device="cuda")
    m.mgs_decode_sh(r.ctx, torch.from_numpy(h).cuda(), md, mv, attrs)
    torch.cuda.synchronize()
    got = attrs.float().cpu().numpy()
    ref = oracle.decode_sh(h.astype(np.float64), md, mv)
    err = np.abs(got[:, 11:23] - ref)
    if prec == "fp32":
        assert err.max() <= 1e-5
    else:
        assert (err <= np.abs(ref) * 2.0 ** -11 + 1e-5).all()
    untouched = np.concatenate([got[:, :11], got[:, 23:]], axis=1)
    assert (untouched == 7.0).all()


def test_decode_then_render(env):
    m, r, torch = env
    n = 30000
    base = synth.unbounded_scene(n, seed=33, precision="fp16").attrs
    md, mv = synth.random_sh_decoders(34)
    h = synth.compressed_sh_features(n, seed=35, precision="fp16")
    attrs = torch.from_numpy(base.copy()).cuda()
    m.mgs_decode_sh(r.ctx, torch.from_numpy(h).cuda(), md, mv, attrs)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 256, 170, 60.0)[2]
    hd = r.load_scene(attrs)
    try:
        img = r.render(hd, cam)["rgb"].cpu().numpy()
    finally:
        r.unload_scene(hd)
    ref_attrs = base.astype(np.float64)
    ref_attrs[:, 11:23] = oracle.decode_sh(h.astype(np.float64), md, mv)
    ref_attrs = ref_attrs.astype(np.float16)     # the scene's storage precision
    ref = oracle.render(ref_attrs, cam)
    assert np.abs(img - ref["rgb"]).max() <= 2e-3


def test_decode_rejects_bad_arguments(env):
    m, r, torch = env
    md, mv = synth.random_sh_decoders(1)
    h = torch.zeros((4, 6), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        m.mgs_decode_sh(r.ctx, h, md, mv, torch.zeros((4, 23), device="cuda"))
    with pytest.raises(TypeError):
        m.mgs_decode_sh(r.ctx, h, md, mv, torch.zeros((4, 24), dtype=torch.float16, device="cuda"))
    bad = synth.SHDecodeMLP(md.w1, md.b1, md.w2[:2], md.b2[:2])
    with pytest.raises(ValueError):
        m.mgs_decode_sh(r.ctx, h, bad, mv, torch.zeros((4, 24), device="cuda"))
