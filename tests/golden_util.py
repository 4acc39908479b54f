"""Loads the JSON fixtures of tests/golden (written by make_golden.py from
the oracle) back into scene, camera and MLP objects."""
import json
import os

import numpy as np

from paper_2603_11531_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ("plain_fp32_37x21", "mlp_fp16_40x24", "sorted_fp32_37x21")


class Cam:
    def __init__(self, d):
        self.R = np.asarray(d["R"], np.float32).reshape(3, 3)
        self.t = np.asarray(d["t"], np.float32)
        self.fx, self.fy, self.cx, self.cy = d["fx"], d["fy"], d["cx"], d["cy"]
        self.width, self.height, self.znear = d["width"], d["height"], d["znear"]


def load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        d = json.load(f)
    dt = np.float16 if d["precision"] == "fp16" else np.float32
    attrs = np.asarray(d["attrs"], np.float64).astype(dt)
    mlp = None
    if d["mlp"] is not None:
        m = d["mlp"]
        mlp = synth.MLPWeights(np.asarray(m["w1"], np.uint16), np.asarray(m["b1"], np.float32),
                               np.asarray(m["w2"], np.uint16), np.asarray(m["b2"], np.float32),
                               np.asarray(m["w3"], np.uint16), np.asarray(m["b3"], np.float32))
    return d, synth.Scene(attrs, mlp), Cam(d["camera"])
