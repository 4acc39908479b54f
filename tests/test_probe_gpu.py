"""Measurement probes (diagnostics, not the render path): the pipe rates and
the scattered-store rate that the bench's roofline divides by come back
finite and within what one SM can do per clock (128 FP32 lanes, 16 MUFU
lanes per SM quarter, one 32-thread store per clock at most)."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_11531_gb300 as mod
    return mod


def test_pipe_rates_are_plausible(m):
    ex2, ffma = m.mgs_probe_rates(0)
    assert math.isfinite(ex2) and 4.0 <= ex2 <= 64.0, ex2
    assert math.isfinite(ffma) and 32.0 <= ffma <= 128.0 * 1.02, ffma


def test_store_rate_is_plausible(m):
    s = m.mgs_probe_store(0)
    assert math.isfinite(s) and 0.05 <= s <= 32.0, s


def test_probes_reject_bad_arguments(m):
    import torch
    for probe in (m.mgs_probe_store, m.mgs_probe_rates):
        with pytest.raises(m.MGSError) as e:
            probe(1 << 20)
        assert e.value.status == m.MGS_ERR_INVALID_ARG
    # the refusal leaves no CUDA error behind for the next render to report
    from paper_2603_11531_gb300 import synth
    r = m.Renderer(0)
    try:
        h = r.load_scene(synth.uniform_scene(64, seed=3, precision="fp32"))
        out = r.render(h, synth.look_at((0, 0, -3), (0, 0, 0), 64, 48, 60.0))
        assert torch.isfinite(out["rgb"]).all()
    finally:
        r.close()
