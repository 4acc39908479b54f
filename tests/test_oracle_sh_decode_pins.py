"""Pins of the oracle's load-time SH decode (Sec. 3.2, Eq. 6) -- CPU only."""
import numpy as np
import pytest

import oracle
from paper_2603_11531_gb300 import synth


def test_half_decode_matches_numpy_for_every_pattern():
    bits = np.arange(65536, dtype=np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.half_to_double(int(b)) for b in bits])
    nan = np.isnan(ref)
    assert (np.isnan(got) == nan).all()
    np.testing.assert_array_equal(got[~nan], ref[~nan])


def test_decode_matches_torch_linear():
    torch = pytest.importorskip("torch")
    md, mv = synth.random_sh_decoders(3)
    h = synth.compressed_sh_features(64, seed=4, precision="fp32").astype(np.float64)

    def net(m):
        f = lambda b: torch.from_numpy(np.asarray(b, np.uint16).view(np.float16).astype(np.float64))
        l1 = torch.nn.Linear(6, 64, dtype=torch.float64)
        l2 = torch.nn.Linear(64, m.w2.shape[0], dtype=torch.float64)
        with torch.no_grad():
            l1.weight.copy_(f(m.w1)); l1.bias.copy_(f(m.b1))
            l2.weight.copy_(f(m.w2)); l2.bias.copy_(f(m.b2))
        return lambda x: l2(torch.relu(l1(x)))

    with torch.no_grad():
        x = torch.from_numpy(h)
        exp = torch.cat([net(md)(x), net(mv)(x)], dim=1).numpy()
    np.testing.assert_allclose(oracle.decode_sh(h, md, mv), exp, rtol=1e-12, atol=1e-12)


def test_zero_weights_give_the_biases_in_sh_order():
    """f_d fills Y0 rgb (columns 0-2), f_v the degree-1 coefficients
    (columns 3-11); with zero weights each output is its bias."""
    md, mv = synth.random_sh_decoders(5)
    for m in (md, mv):
        m.w1 = np.zeros_like(m.w1)
        m.w2 = np.zeros_like(m.w2)
    md.b2 = np.array([1.0, 2.0, 3.0], np.float16).view(np.uint16)
    mv.b2 = np.arange(10, 19, dtype=np.float16).view(np.uint16)
    Y = oracle.decode_sh(np.random.default_rng(1).normal(size=(5, 6)), md, mv)
    expected = [1, 2, 3, 10, 11, 12, 13, 14, 15, 16, 17, 18]
    np.testing.assert_array_equal(Y, np.tile(np.array(expected, np.float64), (5, 1)))
