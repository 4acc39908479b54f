"""Seeded synthetic scenes, cameras and MLP weights for the sort-free renderer.

This module only *generates inputs*.  It holds none of the renderer's arithmetic
(no projection, colour, weighting or compositing); both the CUDA path and the
FP64 oracle consume what it produces, byte for byte.

Record layout (one Gaussian = 24 elements of the stored precision, FP32 or FP16):

    0..2   mean mu (world x, y, z)
    3..5   scale s (activated, > 0), one per local axis
    6..9   rotation quaternion q = (w, x, y, z), NOT normalised (the renderer
           normalises it, Sec. 3.1 treats r_i as a rotation)
    10     opacity o in (0, 1) (activated)
    11..22 first-order SH coefficients Y, coefficient-major:
           Y0(r,g,b), Y1(r,g,b), Y2(r,g,b), Y3(r,g,b)
    23     zero padding (keeps records 16-byte aligned)

The Gaussian parametrisation (mu, Sigma = R S S^T R^T, o, Y) follows App. B; the
degree-1 SH follows Sec. 3.2.  Distributions follow the workload recipes:

* uniform scene:   mu ~ U[-1,1]^3, log s ~ N(-3, 0.5), q ~ N(0,1)^4,
                   o = sigmoid(N(0,1)), Y ~ N(0, 0.3)
* unbounded scene: 80 % of the means uniform in the ellipsoid with radii
                   (4, 2, 4), 20 % on a shell with radius ~ U[30, 60]; the other
                   attributes as above.  This stands in for the Mip-NeRF 360
                   "unbounded" scenes (dense centre, far background), which are
                   not available.

Cameras are world-to-camera (R, t) with OpenCV axes (x right, y down, z forward).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

REC = 24          # elements per Gaussian record
MLP_IN = 22       # [P(3), s(3), q_hat(4), Y(12)]
MLP_HIDDEN = 64
MLP_OUT = 5       # [phi, o, d_r, d_g, d_b]


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # (3, 3) float32, world -> camera, row-major
    t: np.ndarray          # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2

    def as_floats(self) -> np.ndarray:
        """16 float32 values: R (9, row-major), t (3), fx, fy, cx, cy."""
        return np.concatenate([
            np.asarray(self.R, np.float32).reshape(9),
            np.asarray(self.t, np.float32).reshape(3),
            np.array([self.fx, self.fy, self.cx, self.cy], np.float32),
        ]).astype(np.float32)


@dataclasses.dataclass
class MLPWeights:
    """Enhancement MLP parameters (Eq. 4): BF16 weights (as uint16 bit
    patterns, row-major [out][in]) and FP32 biases."""
    w1: np.ndarray   # (64, 22) uint16
    b1: np.ndarray   # (64,) float32
    w2: np.ndarray   # (64, 64) uint16
    b2: np.ndarray   # (64,) float32
    w3: np.ndarray   # (5, 64) uint16, rows: phi, o, d_r, d_g, d_b
    b3: np.ndarray   # (5,) float32
    # three hidden layers (App. C widths): w3 is then the third hidden layer
    # (h3, h2) and w4 (5, h3) the head
    w4: np.ndarray | None = None
    b4: np.ndarray | None = None

    @property
    def hidden(self) -> tuple:
        if self.w4 is None:
            return (self.w1.shape[0], self.w2.shape[0])
        return (self.w1.shape[0], self.w2.shape[0], self.w3.shape[0])


@dataclasses.dataclass
class Scene:
    attrs: np.ndarray                 # (N, 24) float32 or float16
    mlp: MLPWeights | None = None

    @property
    def n(self) -> int:
        return int(self.attrs.shape[0])

    @property
    def precision(self) -> str:
        return "fp16" if self.attrs.dtype == np.float16 else "fp32"


# ----------------------------------------------------------------------------
# BF16 helpers (storage format of the weights; input generation only)
# ----------------------------------------------------------------------------

def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even) and
    return the 16-bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, np.uint16).astype(np.uint32) << 16).view(np.float32)


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------

def _common_attrs(rng: np.random.Generator, n: int) -> np.ndarray:
    a = np.zeros((n, REC), np.float64)
    a[:, 3:6] = np.exp(rng.normal(-3.0, 0.5, size=(n, 3)))
    a[:, 6:10] = rng.normal(0.0, 1.0, size=(n, 4))
    a[:, 10] = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, size=n)))
    a[:, 11:23] = rng.normal(0.0, 0.3, size=(n, 12))
    return a


def _store(a: np.ndarray, precision: str) -> np.ndarray:
    if precision == "fp32":
        return np.ascontiguousarray(a.astype(np.float32))
    if precision == "fp16":
        return np.ascontiguousarray(a.astype(np.float16))
    raise ValueError(precision)


def uniform_scene(n: int, seed: int, precision: str = "fp32") -> Scene:
    """Means uniform in [-1,1]^3; the small-scene recipe."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.uniform(-1.0, 1.0, size=(n, 3))
    a = _common_attrs(rng, n)
    a[:, 0:3] = mu
    return Scene(_store(a, precision))


def unbounded_scene(n: int, seed: int, precision: str = "fp16",
                    inner_frac: float = 0.8) -> Scene:
    """Dense ellipsoid (radii 4, 2, 4) plus a far shell (radius 30..60),
    in generation order: the inner points first, then the shell."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_in = int(round(n * inner_frac))
    n_sh = n - n_in
    d = rng.normal(size=(n_in, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    u = rng.uniform(0.0, 1.0, size=(n_in, 1)) ** (1.0 / 3.0)
    inner = d * u * np.array([4.0, 2.0, 4.0])
    d2 = rng.normal(size=(n_sh, 3))
    d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    shell = d2 * rng.uniform(30.0, 60.0, size=(n_sh, 1))
    a = _common_attrs(rng, n)
    a[:, 0:3] = np.concatenate([inner, shell], axis=0)
    return Scene(_store(a, precision))


def random_mlp(seed: int, hidden=(MLP_HIDDEN, MLP_HIDDEN)) -> MLPWeights:
    """Kaiming-uniform weights (bound sqrt(6/fan_in)) rounded to BF16; hidden
    biases U(-1/sqrt(fan_in), 1/sqrt(fan_in)); head biases (phi, o, rgb) =
    (1, 0, 0, 0, 0) so that phi starts near 1 (Sec. 3.4 initialises MLP_phi
    to output 1).  `hidden` = (64, 64) or three widths such as App. C's
    (256, 128, 64)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def lin(out_f, in_f):
        bound = math.sqrt(6.0 / in_f)
        w = rng.uniform(-bound, bound, size=(out_f, in_f)).astype(np.float32)
        bb = 1.0 / math.sqrt(in_f)
        b = rng.uniform(-bb, bb, size=out_f).astype(np.float32)
        return f32_to_bf16_bits(w), b

    head_b = np.array([1.0, 0.0, 0.0, 0.0, 0.0], np.float32)
    if len(hidden) == 2 and tuple(hidden) == (MLP_HIDDEN, MLP_HIDDEN):
        w1, b1 = lin(MLP_HIDDEN, MLP_IN)
        w2, b2 = lin(MLP_HIDDEN, MLP_HIDDEN)
        w3, _ = lin(MLP_OUT, MLP_HIDDEN)
        return MLPWeights(w1, b1, w2, b2, w3, head_b)
    h1, h2, h3 = (int(h) for h in hidden)
    w1, b1 = lin(h1, MLP_IN)
    w2, b2 = lin(h2, h1)
    w3, b3 = lin(h3, h2)
    w4, _ = lin(MLP_OUT, h3)
    return MLPWeights(w1, b1, w2, b2, w3, b3, w4, head_b)


@dataclasses.dataclass
class SHDecodeMLP:
    """One load-time SH decoder of Eq. 6: 6 -> 64 (ReLU) -> n_out, all
    parameters as IEEE binary16 bit patterns (uint16), row-major [out][in]."""
    w1: np.ndarray   # (64, 6)
    b1: np.ndarray   # (64,)
    w2: np.ndarray   # (n_out, 64)
    b2: np.ndarray   # (n_out,)


def random_sh_decoders(seed: int):
    """(MLP_d with 3 outputs, MLP_v with 9 outputs): Kaiming-uniform FP16
    weights, small FP16 biases."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def mk(n_out):
        b1 = math.sqrt(6.0 / 6)
        w1 = rng.uniform(-b1, b1, size=(64, 6)).astype(np.float16).view(np.uint16)
        bb1 = rng.uniform(-0.1, 0.1, size=64).astype(np.float16).view(np.uint16)
        b2 = math.sqrt(6.0 / 64) * 0.5
        w2 = rng.uniform(-b2, b2, size=(n_out, 64)).astype(np.float16).view(np.uint16)
        bb2 = rng.uniform(-0.1, 0.1, size=n_out).astype(np.float16).view(np.uint16)
        return SHDecodeMLP(w1, bb1, w2, bb2)

    return mk(3), mk(9)


def compressed_sh_features(n: int, seed: int, precision: str = "fp16") -> np.ndarray:
    """Per-Gaussian (h_d, h_v) of Eq. 6 as stored after dequantisation:
    N(0, 0.5) values, (n, 6)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.normal(0.0, 0.5, size=(n, 6)).astype(np.float32)
    return h.astype(np.float16) if precision == "fp16" else h


PAPER_MLP_HIDDEN = (256, 128, 64)   # App. C: MLP_f widths


def random_mlp_paper(seed: int) -> MLPWeights:
    """random_mlp with the paper's MLP_f widths 256, 128, 64 (App. C)."""
    return random_mlp(seed, PAPER_MLP_HIDDEN)


# ----------------------------------------------------------------------------
# Cameras
# ----------------------------------------------------------------------------

def look_at(eye, target, width: int, height: int, fov_x_deg: float,
            znear: float = 0.2) -> Camera:
    """Pinhole camera at `eye` looking at `target`; world 'down' is +y
    (OpenCV convention), principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(R.astype(np.float32), t.astype(np.float32), float(np.float32(fx)),
                  float(np.float32(fx)), float(np.float32(0.5 * width)),
                  float(np.float32(0.5 * height)), int(width), int(height),
                  float(np.float32(znear)))


def orbit_cameras(n_poses: int, radius: float, height_up: float, width: int,
                  height: int, fov_x_deg: float = 60.0) -> list[Camera]:
    """`n_poses` cameras on a horizontal circle of `radius` at `height_up`
    world units above the origin (world up = -y), all looking at the origin;
    pose k sits at angle 2*pi*k/n_poses."""
    cams = []
    for k in range(n_poses):
        th = 2.0 * math.pi * k / n_poses
        eye = (radius * math.sin(th), -height_up, -radius * math.cos(th))
        cams.append(look_at(eye, (0.0, 0.0, 0.0), width, height, fov_x_deg))
    return cams


def random_orbit_camera(rng: np.random.Generator, width: int, height: int,
                        radius: float = 8.0, height_up: float = 1.0,
                        fov_x_deg: float = 60.0) -> Camera:
    th = rng.uniform(0.0, 2.0 * math.pi)
    eye = (radius * math.sin(th), -height_up, -radius * math.cos(th))
    return look_at(eye, (0.0, 0.0, 0.0), width, height, fov_x_deg)


# ----------------------------------------------------------------------------
# The five workload recipes (sizes and seeds fixed)
# ----------------------------------------------------------------------------

def workload_small_fp32():
    """4,096 Gaussians, FP32, one 256x256 camera at distance 3, fov 60 deg."""
    scene = uniform_scene(4096, seed=1, precision="fp32")
    cam = look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 256, 256, 60.0)
    return scene, [cam]


def workload_unbounded_600k(n_poses: int = 64, n: int = 600_000):
    """600k Gaussians, FP16 attributes, BF16 MLP, 1600x1063, orbit poses."""
    scene = unbounded_scene(n, seed=2, precision="fp16")
    scene.mlp = random_mlp(seed=20)
    cams = orbit_cameras(n_poses, 8.0, 1.0, 1600, 1063, 60.0)
    return scene, cams


def workload_backward_300k():
    """300k Gaussians (unbounded distribution), FP32, MLP on, 1296x840."""
    scene = unbounded_scene(300_000, seed=3, precision="fp32")
    scene.mlp = random_mlp(seed=30)
    cam = orbit_cameras(1, 8.0, 1.0, 1296, 840, 60.0)[0]
    rng = np.random.Generator(np.random.PCG64(33))
    target = rng.uniform(0.0, 1.0, size=(840, 1296, 3)).astype(np.float32)
    return scene, cam, target


SERVING_SIZES = (50_000, 90_000, 160_000, 300_000, 550_000, 1_000_000,
                 1_700_000, 3_000_000)
SERVING_RESOLUTIONS = ((640, 480), (1280, 720), (1600, 1063), (1920, 1080))


def serving_scenes(sizes=SERVING_SIZES):
    """Eight resident scenes, unbounded distribution, FP16, seed 40 + k."""
    out = []
    for k, n in enumerate(sizes):
        s = unbounded_scene(n, seed=40 + k, precision="fp16")
        s.mlp = random_mlp(seed=400 + k)
        out.append(s)
    return out


def workload_large_6m():
    """6M Gaussians, FP16, 3840x2160, one orbit pose."""
    scene = unbounded_scene(6_000_000, seed=5, precision="fp16")
    scene.mlp = random_mlp(seed=50)
    cam = orbit_cameras(1, 8.0, 1.0, 3840, 2160, 60.0)[0]
    return scene, cam
