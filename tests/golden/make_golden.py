"""Writes the golden fixtures of this folder from the FP64 oracle (and only
from it): small seeded scenes, their inputs, and the oracle's images,
per-pixel inclusion counts and tile lists, as JSON text.

    python tests/golden/make_golden.py

Each fixture cites the passages it exercises.  The oracle is test
infrastructure; nothing on the GPU path reads these files except the tests.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_11531_gb300 import synth  # noqa: E402


def cam_dict(c):
    return {"R": np.asarray(c.R, np.float64).reshape(9).tolist(), "t": np.asarray(c.t, np.float64).tolist(),
            "fx": float(c.fx), "fy": float(c.fy), "cx": float(c.cx), "cy": float(c.cy),
            "width": int(c.width), "height": int(c.height), "znear": float(getattr(c, "znear", 0.2))}


def mlp_dict(m):
    return {k: np.asarray(getattr(m, k)).tolist() for k in ("w1", "b1", "w2", "b2", "w3", "b3")}


def fixture(name, cite, attrs, cam, bg, mlp=None, use_mlp=False, sorted_=False):
    if sorted_:
        out = oracle.render_sorted(attrs, cam, mlp=mlp, use_mlp=use_mlp, bg=bg, want_count=True)
    else:
        out = oracle.render(attrs, cam, mlp=mlp, use_mlp=use_mlp, bg=bg, want_count=True)
    d = {"name": name, "cite": cite, "precision": "fp16" if attrs.dtype == np.float16 else "fp32",
         "attrs": attrs.astype(np.float64).tolist(), "camera": cam_dict(cam), "bg": list(map(float, bg)),
         "use_mlp": bool(use_mlp), "sorted": bool(sorted_), "mlp": mlp_dict(mlp) if mlp is not None else None,
         "rgb": np.round(out["rgb"], 15).tolist(), "count": out["count"].tolist(),
         "offsets": np.asarray(out["offsets"]).tolist(), "gids": np.asarray(out["gids"]).tolist()}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(d, f)


def main():
    oracle.build()
    a = synth.uniform_scene(48, seed=501).attrs
    fixture("plain_fp32_37x21", "Sec. 3.1 Eq. 2-3, App. B projection; 3 x 2 tiles with ragged edges",
            a, synth.look_at((0.1, 0.0, -2.5), (0, 0, 0), 37, 21, 60.0), (0.05, 0.1, 0.2))
    s = synth.unbounded_scene(160, seed=502, precision="fp16")
    s.mlp = synth.random_mlp(503)
    fixture("mlp_fp16_40x24", "Sec. 3.1 Eq. 2-4 (BF16 MLP), Sec. 3.2 degree-1 SH",
            s.attrs, synth.orbit_cameras(8, 8.0, 1.0, 40, 24, 60.0)[1], (0.0, 0.0, 0.0), s.mlp, True)
    fixture("sorted_fp32_37x21", "App. B Eq. 11: sorted front-to-back comparator",
            a, synth.look_at((0.1, 0.0, -2.5), (0, 0, 0), 37, 21, 60.0), (0.05, 0.1, 0.2), sorted_=True)


if __name__ == "__main__":
    main()
