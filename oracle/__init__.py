"""Python access to the FP64 CPU oracle (``mgs_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It imports nothing from
the CUDA renderer package; scenes and cameras are passed in as plain arrays
and duck-typed objects (attributes ``R, t, fx, fy, cx, cy, width, height,
znear``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgs_oracle.c")
_HDR = os.path.join(_HERE, "mgs_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fno-math-errno", "-Wall", "-Wextra", _SRC,
               "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("znear", ctypes.c_float)]


class _MLP(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p),
                ("w4", ctypes.c_void_p), ("b4", ctypes.c_void_p),
                ("h1", ctypes.c_int32), ("h2", ctypes.c_int32), ("h3", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


GAUSS_DTYPE = np.dtype([
    ("visible", np.int32), ("rect", np.int32, 4), ("m32", np.float32, 2),
    ("l32", np.float32, 3), ("tz32", np.float32), ("mean", np.float64, 2), ("cov", np.float64, 3),
    ("conic", np.float64, 3), ("depth", np.float64), ("rgb", np.float64, 3),
    ("opacity", np.float64), ("phi", np.float64), ("weight", np.float64),
    ("dir", np.float64, 3)], align=True)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.orc_gauss_size.restype = ctypes.c_int64
            L.orc_rotation.argtypes = [P, P]
            L.orc_bf16_round.restype = ctypes.c_double
            L.orc_bf16_round.argtypes = [ctypes.c_double]
            L.orc_mlp_eval.argtypes = [P, P, P]
            L.orc_preprocess.restype = ctypes.c_int
            L.orc_preprocess.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int,
                                         ctypes.c_int, P]
            L.orc_bin.restype = ctypes.c_int64
            L.orc_bin.argtypes = [ctypes.c_int64, P, ctypes.c_int, ctypes.c_int, P,
                                  P, ctypes.c_int64]
            L.orc_tile_may_hit.restype = ctypes.c_int
            L.orc_tile_may_hit.argtypes = [P, ctypes.c_int, ctypes.c_int]
            L.orc_includes.restype = ctypes.c_int
            L.orc_includes.argtypes = [P, ctypes.c_int, ctypes.c_int]
            L.orc_rasterize.restype = ctypes.c_int
            L.orc_rasterize.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int,
                                        ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                        P, P, P]
            L.orc_decode_sh.restype = None
            L.orc_decode_sh.argtypes = [ctypes.c_int64, P, P, P, P]
            L.orc_half_to_double.restype = ctypes.c_double
            L.orc_half_to_double.argtypes = [ctypes.c_uint16]
            L.orc_rasterize_depth.restype = ctypes.c_int
            L.orc_rasterize_depth.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.orc_rasterize_sorted.restype = ctypes.c_int
            L.orc_rasterize_sorted.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int,
                                               ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P]
            L.orc_pairs.restype = ctypes.c_int64
            L.orc_pairs.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int64]
            if L.orc_gauss_size() != GAUSS_DTYPE.itemsize:
                raise RuntimeError("orc_gauss layout mismatch")
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def make_camera(cam) -> _Camera:
    c = _Camera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(np.float32(getattr(cam, "znear", 0.2)))
    return c


class _MLPHolder:
    """Keeps the contiguous weight arrays alive while the C struct points at them."""

    def __init__(self, mlp):
        w4 = getattr(mlp, "w4", None)
        self.arrays = [np.ascontiguousarray(mlp.w1, np.uint16),
                       np.ascontiguousarray(mlp.b1, np.float32),
                       np.ascontiguousarray(mlp.w2, np.uint16),
                       np.ascontiguousarray(mlp.b2, np.float32),
                       np.ascontiguousarray(mlp.w3, np.uint16),
                       np.ascontiguousarray(mlp.b3, np.float32)]
        if w4 is None:
            assert self.arrays[0].shape == (64, 22) and self.arrays[2].shape == (64, 64)
            assert self.arrays[4].shape == (5, 64)
            dims = (0, 0, 0)
            self.arrays += [None, None]
        else:
            h1, h2, h3 = self.arrays[0].shape[0], self.arrays[2].shape[0], self.arrays[4].shape[0]
            assert self.arrays[0].shape == (h1, 22) and self.arrays[2].shape == (h2, h1)
            assert self.arrays[4].shape == (h3, h2) and np.shape(w4) == (5, h3)
            assert max(h1, h2, h3) <= 256
            dims = (h1, h2, h3)
            self.arrays += [np.ascontiguousarray(w4, np.uint16),
                            np.ascontiguousarray(mlp.b4, np.float32)]
        ptrs = [a.ctypes.data if a is not None else None for a in self.arrays]
        self.s = _MLP(*ptrs, *dims, 0)


def tiles(width: int, height: int) -> tuple[int, int]:
    return (width + TILE - 1) // TILE, (height + TILE - 1) // TILE


def preprocess(attrs: np.ndarray, cam, mlp=None, use_mlp: bool = False,
               rgb_residual: bool = False) -> np.ndarray:
    """App. B projection + Sec. 3.2 colour + Eq. 3/4 for every Gaussian.
    Returns a structured array (GAUSS_DTYPE)."""
    a64 = np.ascontiguousarray(np.asarray(attrs).astype(np.float64))
    assert a64.ndim == 2 and a64.shape[1] == 24
    n = a64.shape[0]
    out = np.zeros(n, GAUSS_DTYPE)
    c = make_camera(cam)
    holder = _MLPHolder(mlp) if (use_mlp and mlp is not None) else None
    rc = lib().orc_preprocess(n, _ptr(a64), ctypes.byref(c),
                              ctypes.byref(holder.s) if holder else None,
                              int(bool(use_mlp)), int(bool(rgb_residual)), _ptr(out))
    if rc != 0:
        raise ValueError("orc_preprocess failed (MLP requested without weights?)")
    return out


def bin_tiles(g: np.ndarray, width: int, height: int):
    """Per-tile Gaussian lists (ascending index), no depth order."""
    tx, ty = tiles(width, height)
    offsets = np.zeros(tx * ty + 1, np.int64)
    K = lib().orc_bin(len(g), _ptr(g), tx, ty, _ptr(offsets), None, 0)
    gids = np.zeros(max(K, 1), np.int32)
    K2 = lib().orc_bin(len(g), _ptr(g), tx, ty, _ptr(offsets), _ptr(gids), K)
    assert K2 == K
    return offsets, gids[:K]


def rasterize(g: np.ndarray, offsets, gids, width: int, height: int, bg=(0.0, 0.0, 0.0),
              tile_range=None, want_aux: bool = False, want_count: bool = False):
    """Eq. 2 per pixel.  Returns (rgb HxWx3, aux 5xHxW | None, count HxW | None)."""
    tx, ty = tiles(width, height)
    t0, t1 = (0, tx * ty) if tile_range is None else tile_range
    rgb = np.zeros((height, width, 3), np.float64)
    aux = np.zeros((5, height, width), np.float64) if want_aux else None
    cnt = np.zeros((height, width), np.int32) if want_count else None
    bgv = np.ascontiguousarray(np.asarray(bg, np.float64).reshape(3))
    gids = np.ascontiguousarray(gids, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    lib().orc_rasterize(len(g), _ptr(g), _ptr(offsets), _ptr(gids if len(gids) else np.zeros(1, np.int32)),
                        width, height, _ptr(bgv), t0, t1, _ptr(rgb), _ptr(aux), _ptr(cnt))
    return rgb, aux, cnt


def render(attrs, cam, mlp=None, use_mlp=False, rgb_residual=False, bg=(0.0, 0.0, 0.0),
           want_aux=False, want_count=False, tile_range=None):
    """Whole forward path: preprocess -> bin -> rasterize."""
    g = preprocess(attrs, cam, mlp, use_mlp, rgb_residual)
    offsets, gids = bin_tiles(g, cam.width, cam.height)
    rgb, aux, cnt = rasterize(g, offsets, gids, cam.width, cam.height, bg, tile_range,
                              want_aux, want_count)
    return dict(gauss=g, offsets=offsets, gids=gids, rgb=rgb, aux=aux, count=cnt)


def rasterize_depth(g: np.ndarray, offsets, gids, width: int, height: int, tile_range=None):
    """Depth image for Eq. 5: D = sum d a w / sum a w per pixel (0 if empty)."""
    tx, ty = tiles(width, height)
    t0, t1 = (0, tx * ty) if tile_range is None else tile_range
    depth = np.zeros((height, width), np.float64)
    gids = np.ascontiguousarray(gids, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    lib().orc_rasterize_depth(len(g), _ptr(g), _ptr(offsets),
                              _ptr(gids if len(gids) else np.zeros(1, np.int32)),
                              width, height, t0, t1, _ptr(depth))
    return depth


def render_depth(attrs, cam, mlp=None, use_mlp=False, rgb_residual=False, tile_range=None):
    """preprocess -> bin -> depth image (Sec. 3.2, Eq. 5)."""
    g = preprocess(attrs, cam, mlp, use_mlp, rgb_residual)
    offsets, gids = bin_tiles(g, cam.width, cam.height)
    return dict(gauss=g, offsets=offsets, gids=gids,
                depth=rasterize_depth(g, offsets, gids, cam.width, cam.height, tile_range))


class _SHMLP(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p),
                ("b2", ctypes.c_void_p), ("n_out", ctypes.c_int32), ("pad", ctypes.c_int32)]


def decode_sh(h, mlp_d, mlp_v) -> np.ndarray:
    """Eq. 6 load-time decode: h (n, 6) = (h_d, h_v) -> SH coefficients (n, 12),
    [f_d (Y0 rgb), f_v (Y1 rgb, Y2 rgb, Y3 rgb)].  mlp_*: objects with w1, b1,
    w2, b2 as binary16 bit patterns (uint16)."""
    h = np.ascontiguousarray(h, np.float64).reshape(-1, 6)
    keep, structs = [], []
    for m, n_out in ((mlp_d, 3), (mlp_v, 9)):
        arrs = [np.ascontiguousarray(getattr(m, k), np.uint16) for k in ("w1", "b1", "w2", "b2")]
        assert arrs[0].shape == (64, 6) and arrs[1].shape == (64,)
        assert arrs[2].shape == (n_out, 64) and arrs[3].shape == (n_out,)
        keep += arrs
        structs.append(_SHMLP(*[a.ctypes.data for a in arrs], n_out, 0))
    Y = np.zeros((len(h), 12), np.float64)
    if len(h):
        lib().orc_decode_sh(len(h), _ptr(h), ctypes.byref(structs[0]), ctypes.byref(structs[1]),
                            _ptr(Y))
    return Y


def half_to_double(bits: int) -> float:
    return lib().orc_half_to_double(int(bits))


def rotation(q) -> np.ndarray:
    q = np.ascontiguousarray(np.asarray(q, np.float64).reshape(4))
    R = np.zeros(9, np.float64)
    lib().orc_rotation(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def bf16_round(v: float) -> float:
    return lib().orc_bf16_round(float(v))


def mlp_eval(mlp, x) -> np.ndarray:
    holder = _MLPHolder(mlp)
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(22))
    out = np.zeros(5, np.float64)
    lib().orc_mlp_eval(ctypes.byref(holder.s), _ptr(x), _ptr(out))
    return out


def includes(g_row: np.ndarray, px: int, py: int) -> bool:
    one = np.ascontiguousarray(np.asarray(g_row).reshape(1))
    return bool(lib().orc_includes(_ptr(one), int(px), int(py)))


def tile_may_hit(g_row: np.ndarray, tx: int, ty: int) -> bool:
    one = np.ascontiguousarray(np.asarray(g_row).reshape(1))
    return bool(lib().orc_tile_may_hit(_ptr(one), int(tx), int(ty)))


def included_pairs(g: np.ndarray, offsets, gids, width: int, height: int):
    """(pixel_index, gaussian_index) of every included pair (FP32 contract)."""
    offsets = np.ascontiguousarray(offsets, np.int64)
    gids = np.ascontiguousarray(gids, np.int32)
    gp = _ptr(gids if len(gids) else np.zeros(1, np.int32))
    n = lib().orc_pairs(_ptr(g), _ptr(offsets), gp, width, height, None, None, 0)
    pix = np.zeros(max(n, 1), np.int64)
    gid = np.zeros(max(n, 1), np.int32)
    n2 = lib().orc_pairs(_ptr(g), _ptr(offsets), gp, width, height, _ptr(pix), _ptr(gid), n)
    assert n2 == n
    return pix[:n], gid[:n]


def rasterize_sorted(g: np.ndarray, offsets, gids, width: int, height: int,
                     bg=(0.0, 0.0, 0.0), tile_range=None, want_count: bool = False):
    """Comparator: sorted front-to-back alpha blending (App. B, Eq. 11)."""
    tx, ty = tiles(width, height)
    t0, t1 = (0, tx * ty) if tile_range is None else tile_range
    rgb = np.zeros((height, width, 3), np.float64)
    cnt = np.zeros((height, width), np.int32) if want_count else None
    bgv = np.ascontiguousarray(np.asarray(bg, np.float64).reshape(3))
    gids = np.ascontiguousarray(gids, np.int32)
    offsets = np.ascontiguousarray(offsets, np.int64)
    rc = lib().orc_rasterize_sorted(len(g), _ptr(g), _ptr(offsets),
                                    _ptr(gids if len(gids) else np.zeros(1, np.int32)),
                                    width, height, _ptr(bgv), t0, t1, _ptr(rgb), _ptr(cnt))
    if rc != 0:
        raise MemoryError("orc_rasterize_sorted")
    return rgb, cnt


def render_sorted(attrs, cam, mlp=None, use_mlp=False, rgb_residual=False, bg=(0.0, 0.0, 0.0),
                  want_count=False, tile_range=None):
    g = preprocess(attrs, cam, mlp, use_mlp, rgb_residual)
    offsets, gids = bin_tiles(g, cam.width, cam.height)
    rgb, cnt = rasterize_sorted(g, offsets, gids, cam.width, cam.height, bg, tile_range, want_count)
    return dict(gauss=g, offsets=offsets, gids=gids, rgb=rgb, count=cnt)
