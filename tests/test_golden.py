"""The oracle reproduces the committed golden fixtures (tests/golden, written
by make_golden.py from the oracle): a regression pin on the oracle itself.
CPU only."""
import numpy as np
import pytest

import oracle
from golden_util import NAMES, load


@pytest.mark.parametrize("name", NAMES)
def test_oracle_reproduces_fixture(name):
    d, scene, cam = load(name)
    kw = dict(mlp=scene.mlp, use_mlp=d["use_mlp"], bg=d["bg"], want_count=True)
    out = oracle.render_sorted(scene.attrs, cam, **kw) if d["sorted"] else oracle.render(scene.attrs, cam, **kw)
    np.testing.assert_allclose(out["rgb"], np.asarray(d["rgb"]), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(out["count"], np.asarray(d["count"]))
    np.testing.assert_array_equal(np.asarray(out["offsets"]), np.asarray(d["offsets"]))
    np.testing.assert_array_equal(np.asarray(out["gids"]), np.asarray(d["gids"]))
