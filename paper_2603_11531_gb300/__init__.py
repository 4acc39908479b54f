"""Python binding of the GB300 sort-free Gaussian renderer (libmobilegs.so).

Argument marshalling only: every step of a render runs in the CUDA kernels
behind the C-ABI (include/mobilegs.h).  The functions mirror the C entry
points by name; `Renderer` bundles a context, a workspace and torch output
buffers for convenience.  There is no CPU fallback: if the compiled library
is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmobilegs.so")
_lib = None
_lock = threading.Lock()

MGS_OK = 0
MGS_ERR_INVALID_ARG = 1
MGS_ERR_OOM = 2
MGS_ERR_CUDA = 3
MGS_ERR_OVERFLOW = 4
MGS_ERR_TIMEOUT = 5
MGS_ERR_BUSY = 6
MGS_ERR_NOT_READY = 7
MGS_PREC_FP32 = 0
MGS_PREC_FP16 = 1
MGS_FLAG_NO_CULL = 1
MGS_FLAG_SORTED = 2
MGS_FLAG_MLP_MMA_SYNC = 4
MGS_FLAG_RASTER_FMA = 8
MGS_ORDER_AUTO = 0
MGS_ORDER_SPATIAL = 1
MGS_ORDER_AS_GIVEN = 2

# Every entry point declared in include/mobilegs.h.
EXPORTS = (
    "mgs_ctx_create", "mgs_ctx_destroy", "mgs_ctx_info", "mgs_load_scene",
    "mgs_unload_scene", "mgs_scene_bytes", "mgs_workspace_create", "mgs_workspace_destroy",
    "mgs_workspace_reserve", "mgs_workspace_bytes", "mgs_workspace_sync", "mgs_render",
    "mgs_render_checked", "mgs_render_to_host", "mgs_tile_lists", "mgs_last_error",
    "mgs_version", "mgs_workspace_set_timing", "mgs_workspace_stage_times",
    "mgs_render_static", "mgs_render_backward", "mgs_render_depth", "mgs_decode_sh",
    "mgs_server_create", "mgs_server_destroy", "mgs_server_submit", "mgs_server_wait",
    "mgs_server_ticket", "mgs_server_stats", "mgs_now", "mgs_probe_rates", "mgs_probe_store", "mgs_frame_stats",
)
MLP_GRAD_SIZE = 5957


class MGSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mobilegs status {status}: {msg}")
        self.status = status


class mgs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("znear", ctypes.c_float)]


class mgs_render_opts(ctypes.Structure):
    _fields_ = [("use_mlp", ctypes.c_int32), ("mlp_rgb_residual", ctypes.c_int32),
                ("bg", ctypes.c_float * 3), ("flags", ctypes.c_uint32)]


class mgs_scene_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("attrs_on_device", ctypes.c_int32), ("attrs", ctypes.c_void_p),
                ("mlp_w1", ctypes.c_void_p), ("mlp_b1", ctypes.c_void_p),
                ("mlp_w2", ctypes.c_void_p), ("mlp_b2", ctypes.c_void_p),
                ("mlp_w3", ctypes.c_void_p), ("mlp_b3", ctypes.c_void_p),
                ("mlp_w4", ctypes.c_void_p), ("mlp_b4", ctypes.c_void_p),
                ("mlp_hidden", ctypes.c_int32 * 3), ("order", ctypes.c_int32)]


class mgs_sh_mlp(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p)]


def lib():
    """Load libmobilegs.so (built by build.py / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            PP = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "mgs_ctx_create": ([I32, PP], I32),
                "mgs_ctx_destroy": ([P], I32),
                "mgs_ctx_info": ([P, ctypes.POINTER(I32), ctypes.POINTER(I64), ctypes.POINTER(I64)], I32),
                "mgs_load_scene": ([P, ctypes.POINTER(mgs_scene_desc), P, PP], I32),
                "mgs_unload_scene": ([P], I32),
                "mgs_scene_bytes": ([P], I64),
                "mgs_workspace_create": ([P, PP], I32),
                "mgs_workspace_destroy": ([P], I32),
                "mgs_workspace_reserve": ([P, I64, I32, I32, I64], I32),
                "mgs_workspace_bytes": ([P], I64),
                "mgs_workspace_sync": ([P, P, ctypes.POINTER(I64)], I32),
                "mgs_render": ([P, P, ctypes.POINTER(mgs_camera), ctypes.POINTER(mgs_render_opts),
                                P, P, P, P], I32),
                "mgs_render_checked": ([P, P, ctypes.POINTER(mgs_camera),
                                        ctypes.POINTER(mgs_render_opts), P, P, P, P], I32),
                "mgs_render_to_host": ([P, P, ctypes.POINTER(mgs_camera),
                                        ctypes.POINTER(mgs_render_opts), P, P], I32),
                "mgs_render_depth": ([P, P, ctypes.POINTER(mgs_camera),
                                      ctypes.POINTER(mgs_render_opts), P, P, P], I32),
                "mgs_tile_lists": ([P, P, ctypes.POINTER(I64), ctypes.POINTER(I64), P, P], I32),
                "mgs_frame_stats": ([P, P, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                     ctypes.POINTER(I64)], I32),
                "mgs_workspace_set_timing": ([P, I32], I32),
                "mgs_workspace_stage_times": ([P, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)], I32),
                "mgs_render_static": ([P, I64, I32, ctypes.POINTER(mgs_camera),
                                       ctypes.POINTER(mgs_render_opts), P, P], I32),
                "mgs_render_backward": ([P, P, ctypes.POINTER(mgs_camera),
                                         ctypes.POINTER(mgs_render_opts), P, P, P, P, P], I32),
                "mgs_decode_sh": ([P, I64, I32, P, ctypes.POINTER(mgs_sh_mlp),
                                   ctypes.POINTER(mgs_sh_mlp), P, P], I32),
                "mgs_probe_rates": ([I32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)], I32),
                "mgs_probe_store": ([I32, ctypes.POINTER(ctypes.c_double)], I32),
                "mgs_last_error": ([], ctypes.c_char_p),
                "mgs_version": ([], ctypes.c_char_p),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(status: int, allow=()) -> int:
    if status != MGS_OK and status not in allow:
        raise MGSError(status, lib().mgs_last_error().decode())
    return status


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream, device=None) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream(device).cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# CUDA device of every context, workspace and loaded scene created through
# this module (keyed by handle value), and each scene's Gaussian count, so
# that output buffers can be checked before the library writes through them.
_ctx_dev: dict = {}
_ws_dev: dict = {}
_scene_info: dict = {}


def _dev_of(handle, table, what):
    v = getattr(handle, "value", handle)
    if v not in table:
        raise ValueError(f"unknown {what} handle (not created through this module)")
    return table[v]


def _check_dev_tensor(t, shape, dtype, device, what, optional=False):
    """Raise ValueError unless t is a contiguous CUDA tensor of `shape` and
    `dtype` on CUDA device `device` (None allowed when optional)."""
    import torch
    if t is None:
        if optional:
            return
        raise ValueError(f"{what} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if device is not None and t.device.index != device:
        raise ValueError(f"{what} is on cuda:{t.device.index}, the call runs on cuda:{device}")


def _check_host_buffer(t, shape, what):
    """Raise ValueError unless t is a contiguous float32 host buffer (CPU
    tensor or numpy array) of `shape`."""
    import torch
    if isinstance(t, torch.Tensor):
        ok = (not t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
              and tuple(t.shape) == tuple(shape))
    else:
        ok = (isinstance(t, np.ndarray) and t.dtype == np.float32 and t.flags.c_contiguous
              and tuple(t.shape) == tuple(shape))
    if not ok:
        raise ValueError(f"{what} must be a contiguous float32 host buffer of shape {tuple(shape)}")


def _check_render_outputs(ws, cam, out_rgb, out_aux=None, out_count=None, out_depth=None,
                          rgb_optional=False):
    import torch
    dev = _dev_of(ws, _ws_dev, "workspace")
    H, W = int(cam.height), int(cam.width)
    _check_dev_tensor(out_rgb, (H, W, 3), torch.float32, dev, "out_rgb", rgb_optional)
    _check_dev_tensor(out_aux, (5, H, W), torch.float32, dev, "out_aux", True)
    _check_dev_tensor(out_count, (H, W), torch.int32, dev, "out_count", True)
    _check_dev_tensor(out_depth, (H, W), torch.float32, dev, "out_depth", True)
    return dev


def camera_struct(cam) -> mgs_camera:
    c = mgs_camera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = (float(v) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(getattr(cam, "znear", 0.2))
    return c


def render_opts(use_mlp=False, rgb_residual=False, bg=(0.0, 0.0, 0.0), flags=0) -> mgs_render_opts:
    o = mgs_render_opts()
    o.use_mlp = int(bool(use_mlp))
    o.mlp_rgb_residual = int(bool(rgb_residual))
    for k in range(3):
        o.bg[k] = float(bg[k])
    o.flags = int(flags)
    return o


# ---- thin wrappers with the C names ------------------------------------------

def mgs_ctx_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(lib().mgs_ctx_create(device, ctypes.byref(h)))
    _ctx_dev[h.value] = int(device)
    return h


def mgs_ctx_destroy(ctx):
    _check(lib().mgs_ctx_destroy(ctx))
    _ctx_dev.pop(getattr(ctx, "value", ctx), None)


def mgs_ctx_info(ctx):
    sm, fr, tot = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().mgs_ctx_info(ctx, ctypes.byref(sm), ctypes.byref(fr), ctypes.byref(tot)))
    return sm.value, fr.value, tot.value


def mgs_load_scene(ctx, attrs, mlp=None, stream=None, order=MGS_ORDER_AUTO):
    """attrs: (N, 24) float32/float16 numpy array or CUDA torch tensor;
    order: MGS_ORDER_* storage order (images and indices do not depend on it)."""
    d = mgs_scene_desc()
    d.order = int(order)
    keep = []
    on_dev = hasattr(attrs, "is_cuda") and attrs.is_cuda
    if on_dev:
        import torch
        a = attrs.contiguous()
        prec = MGS_PREC_FP16 if a.dtype == torch.float16 else MGS_PREC_FP32
        if a.dtype not in (torch.float16, torch.float32):
            raise TypeError("attrs must be float16 or float32")
    else:
        a = np.ascontiguousarray(attrs)
        if a.dtype not in (np.float16, np.float32):
            raise TypeError("attrs must be float16 or float32")
        prec = MGS_PREC_FP16 if a.dtype == np.float16 else MGS_PREC_FP32
    if a.ndim != 2 or a.shape[1] != 24:
        raise ValueError("attrs must have shape (N, 24)")
    keep.append(a)
    d.n = int(a.shape[0])
    d.precision = prec
    d.attrs_on_device = int(on_dev)
    d.attrs = _ptr(a)
    if mlp is not None:
        arrs = [np.ascontiguousarray(mlp.w1, np.uint16), np.ascontiguousarray(mlp.b1, np.float32),
                np.ascontiguousarray(mlp.w2, np.uint16), np.ascontiguousarray(mlp.b2, np.float32),
                np.ascontiguousarray(mlp.w3, np.uint16), np.ascontiguousarray(mlp.b3, np.float32)]
        w4 = getattr(mlp, "w4", None)
        if w4 is None:
            assert arrs[0].shape == (64, 22) and arrs[2].shape == (64, 64) and arrs[4].shape == (5, 64)
        else:
            arrs += [np.ascontiguousarray(w4, np.uint16), np.ascontiguousarray(mlp.b4, np.float32)]
            h1, h2, h3 = arrs[0].shape[0], arrs[2].shape[0], arrs[4].shape[0]
            d.mlp_hidden[0], d.mlp_hidden[1], d.mlp_hidden[2] = h1, h2, h3
            d.mlp_w4, d.mlp_b4 = arrs[6].ctypes.data, arrs[7].ctypes.data
        keep += arrs
        (d.mlp_w1, d.mlp_b1, d.mlp_w2, d.mlp_b2, d.mlp_w3, d.mlp_b3) = [x.ctypes.data for x in arrs[:6]]
    dev = _dev_of(ctx, _ctx_dev, "context")
    if on_dev and a.device.index != dev:
        raise ValueError(f"attrs is on cuda:{a.device.index}, the context on cuda:{dev}")
    h = ctypes.c_void_p()
    _check(lib().mgs_load_scene(ctx, ctypes.byref(d), _stream(stream, dev), ctypes.byref(h)))
    _scene_info[h.value] = (dev, d.n)
    return h


def mgs_unload_scene(scene):
    _check(lib().mgs_unload_scene(scene))
    _scene_info.pop(getattr(scene, "value", scene), None)


def mgs_scene_bytes(scene) -> int:
    return lib().mgs_scene_bytes(scene)


def mgs_workspace_create(ctx):
    h = ctypes.c_void_p()
    dev = _dev_of(ctx, _ctx_dev, "context")
    _check(lib().mgs_workspace_create(ctx, ctypes.byref(h)))
    _ws_dev[h.value] = dev
    return h


def mgs_workspace_destroy(ws):
    _check(lib().mgs_workspace_destroy(ws))
    _ws_dev.pop(getattr(ws, "value", ws), None)


def mgs_workspace_reserve(ws, n, width, height, pairs):
    _check(lib().mgs_workspace_reserve(ws, int(n), int(width), int(height), int(pairs)))


def mgs_workspace_bytes(ws) -> int:
    return lib().mgs_workspace_bytes(ws)


def mgs_workspace_sync(ws, stream=None, allow_overflow=False):
    pairs = ctypes.c_int64()
    st = lib().mgs_workspace_sync(ws, _stream(stream, _ws_dev.get(getattr(ws, "value", ws))),
                                  ctypes.byref(pairs))
    _check(st, allow=(MGS_ERR_OVERFLOW,) if allow_overflow else ())
    return st, pairs.value


def mgs_render(ws, scene, cam, opts, out_rgb, out_aux=None, out_count=None, stream=None):
    """out_rgb (H, W, 3) float32, out_aux (5, H, W) float32 and out_count
    (H, W) int32: contiguous CUDA tensors on the workspace's device (checked
    here, before the library writes through them)."""
    c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
    dev = _check_render_outputs(ws, c, out_rgb, out_aux, out_count)
    _check(lib().mgs_render(ws, scene, ctypes.byref(c), ctypes.byref(opts), _ptr(out_rgb),
                            _ptr(out_aux), _ptr(out_count), _stream(stream, dev)))


def mgs_render_checked(ws, scene, cam, opts, out_rgb, out_aux=None, out_count=None, stream=None):
    c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
    dev = _check_render_outputs(ws, c, out_rgb, out_aux, out_count)
    _check(lib().mgs_render_checked(ws, scene, ctypes.byref(c), ctypes.byref(opts), _ptr(out_rgb),
                                    _ptr(out_aux), _ptr(out_count), _stream(stream, dev)))


def mgs_render_depth(ws, scene, cam, opts, out_rgb, out_depth, stream=None):
    c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
    if out_depth is None:
        raise ValueError("out_depth is required")
    dev = _check_render_outputs(ws, c, out_rgb, out_depth=out_depth)
    _check(lib().mgs_render_depth(ws, scene, ctypes.byref(c), ctypes.byref(opts), _ptr(out_rgb),
                                  _ptr(out_depth), _stream(stream, dev)))


def mgs_decode_sh(ctx, h, mlp_d, mlp_v, attrs, stream=None):
    """Eq. 6 load-time SH decode into columns 11..22 of the device tensor
    attrs (N, 24); h: device tensor (N, 6) of the same dtype; mlp_*: objects
    with w1, b1, w2, b2 as binary16 bit patterns."""
    import torch
    if attrs.dtype != h.dtype or attrs.dtype not in (torch.float16, torch.float32):
        raise TypeError("h and attrs must both be float16 or float32")
    if not (attrs.is_cuda and h.is_cuda and attrs.is_contiguous() and h.is_contiguous()):
        raise ValueError("h and attrs must be contiguous CUDA tensors")
    if attrs.device != h.device or attrs.device.index != _dev_of(ctx, _ctx_dev, "context"):
        raise ValueError("h, attrs and the context must be on the same device")
    if h.shape[1] != 6 or attrs.shape[1] != 24 or h.shape[0] != attrs.shape[0]:
        raise ValueError("h must be (N, 6) and attrs (N, 24)")
    keep, ss = [], []
    for m, n_out in ((mlp_d, 3), (mlp_v, 9)):
        arrs = [np.ascontiguousarray(getattr(m, k), np.uint16) for k in ("w1", "b1", "w2", "b2")]
        if arrs[0].shape != (64, 6) or arrs[2].shape != (n_out, 64):
            raise ValueError("SH decoder shapes: w1 (64, 6), w2 (%d, 64)" % n_out)
        keep += arrs
        ss.append(mgs_sh_mlp(*[a.ctypes.data for a in arrs]))
    prec = MGS_PREC_FP16 if attrs.dtype == torch.float16 else MGS_PREC_FP32
    _check(lib().mgs_decode_sh(ctx, int(h.shape[0]), prec, _ptr(h), ctypes.byref(ss[0]),
                               ctypes.byref(ss[1]), _ptr(attrs), _stream(stream, attrs.device.index)))


def mgs_render_to_host(ws, scene, cam, opts, host_rgb, stream=None):
    """host_rgb: contiguous float32 host buffer (H, W, 3) (pinned for an
    asynchronous copy)."""
    c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
    dev = _dev_of(ws, _ws_dev, "workspace")
    _check_host_buffer(host_rgb, (int(c.height), int(c.width), 3), "host_rgb")
    _check(lib().mgs_render_to_host(ws, scene, ctypes.byref(c), ctypes.byref(opts),
                                    _ptr(host_rgb), _stream(stream, dev)))


def mgs_tile_lists(ws, offsets_out=None, gids_out=None, stream=None):
    """(n_tiles, n_pairs) of the workspace's last render; copies the lists
    into the given device tensors when both are passed."""
    n, k = ctypes.c_int64(), ctypes.c_int64()
    dev = _dev_of(ws, _ws_dev, "workspace")
    if offsets_out is not None or gids_out is not None:
        import torch
        _check(lib().mgs_tile_lists(ws, _stream(stream, dev), ctypes.byref(n), ctypes.byref(k),
                                    None, None))
        _check_dev_tensor(offsets_out, (n.value + 1,), offsets_out.dtype
                          if offsets_out is not None and offsets_out.dtype in (torch.int32, torch.uint32)
                          else torch.int32, dev, "offsets_out")
        if (gids_out is None or not isinstance(gids_out, torch.Tensor) or gids_out.ndim != 1
                or gids_out.shape[0] < k.value):
            raise ValueError(f"gids_out must be a 1-D CUDA int32 tensor of at least {k.value} entries")
        _check_dev_tensor(gids_out, tuple(gids_out.shape), torch.int32, dev, "gids_out")
    _check(lib().mgs_tile_lists(ws, _stream(stream, dev), ctypes.byref(n), ctypes.byref(k),
                                _ptr(offsets_out), _ptr(gids_out)))
    return n.value, k.value


def mgs_frame_stats(ws, stream=None) -> dict:
    """Visible Gaussians, listed pairs and FP32-sum tiles of the last render."""
    v, k, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().mgs_frame_stats(ws, _stream(stream, _dev_of(ws, _ws_dev, "workspace")),
                                 ctypes.byref(v), ctypes.byref(k), ctypes.byref(t)))
    return {"visible": v.value, "pairs": k.value, "wide_tiles": t.value}


def mgs_workspace_set_timing(ws, enable: bool):
    _check(lib().mgs_workspace_set_timing(ws, int(bool(enable))))


def mgs_workspace_stage_times(ws, stream=None):
    """(ms[6], frames): summed times of preprocess+MLP, binning plan, tile
    count, tile scan, list scatter and rasterise."""
    ms = (ctypes.c_double * 6)()
    fr = ctypes.c_int64()
    _check(lib().mgs_workspace_stage_times(ws, _stream(stream, _dev_of(ws, _ws_dev, "workspace")),
                                           ms, ctypes.byref(fr)))
    return [ms[k] for k in range(6)], fr.value


def mgs_render_static(attrs, cam, opts, out_rgb, stream=None):
    """Allocation-free render (see include/mobilegs.h): attrs is a CUDA tensor
    (N, 24) float32/float16; waits for the stream before returning."""
    import torch
    if not (hasattr(attrs, "is_cuda") and attrs.is_cuda):
        raise TypeError("attrs must be a CUDA tensor")
    if attrs.dtype not in (torch.float16, torch.float32) or attrs.ndim != 2 or attrs.shape[1] != 24:
        raise ValueError("attrs must be (N, 24) float16/float32")
    a = attrs.contiguous()
    prec = MGS_PREC_FP16 if a.dtype == torch.float16 else MGS_PREC_FP32
    c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
    dev = a.device.index
    _check_dev_tensor(out_rgb, (int(c.height), int(c.width), 3), torch.float32, dev, "out_rgb")
    with torch.cuda.device(dev):     # the entry point works on the current device
        _check(lib().mgs_render_static(_ptr(a), int(a.shape[0]), prec, ctypes.byref(c),
                                       ctypes.byref(opts), _ptr(out_rgb), _stream(stream, dev)))


def mgs_render_backward(ws, scene, cam, opts, dL_drgb, aux, d_attrs, d_mlp=None, stream=None):
    """Adjoint of mgs_render (see include/mobilegs.h); device tensors in/out."""
    import torch
    c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
    dev = _dev_of(ws, _ws_dev, "workspace")
    H, W = int(c.height), int(c.width)
    sdev, n = _dev_of(scene, _scene_info, "scene")
    if sdev != dev:
        raise ValueError("scene and workspace are on different devices")
    _check_dev_tensor(dL_drgb, (H, W, 3), torch.float32, dev, "dL_drgb")
    _check_dev_tensor(aux, (5, H, W), torch.float32, dev, "aux")
    _check_dev_tensor(d_attrs, (n, 24), torch.float32, dev, "d_attrs")
    _check_dev_tensor(d_mlp, (MLP_GRAD_SIZE,), torch.float32, dev, "d_mlp", True)
    _check(lib().mgs_render_backward(ws, scene, ctypes.byref(c), ctypes.byref(opts),
                                     _ptr(dL_drgb), _ptr(aux), _ptr(d_attrs), _ptr(d_mlp),
                                     _stream(stream, dev)))


def mgs_probe_rates(device: int = 0):
    """(ex2 per SM per clock, FP32 FFMA per SM per clock), measured."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().mgs_probe_rates(int(device), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mgs_probe_store(device: int = 0):
    """Scattered 4-byte stores (one 32-byte sector each) per SM per clock, measured."""
    a = ctypes.c_double()
    _check(lib().mgs_probe_store(int(device), ctypes.byref(a)))
    return a.value


def mgs_version() -> str:
    return lib().mgs_version().decode()


# ---- convenience -------------------------------------------------------------

class Renderer:
    """One context + one workspace on a CUDA device; outputs are torch tensors."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = mgs_ctx_create(device)
        self.ws = mgs_workspace_create(self.ctx)
        self._scenes = []

    def load_scene(self, scene_or_attrs, mlp=None, stream=None, order=MGS_ORDER_AUTO):
        attrs = getattr(scene_or_attrs, "attrs", scene_or_attrs)
        if mlp is None:
            mlp = getattr(scene_or_attrs, "mlp", None)
        h = mgs_load_scene(self.ctx, attrs, mlp, stream, order)
        self._scenes.append(h)
        return h

    def unload_scene(self, h):
        mgs_unload_scene(h)
        self._scenes = [s for s in self._scenes if s.value != h.value]

    def render(self, scene, cam, use_mlp=False, rgb_residual=False, bg=(0.0, 0.0, 0.0),
               aux=False, count=False, flags=0, stream=None, checked=True):
        torch = self.torch
        dev = torch.device("cuda", self.device)
        H, W = int(cam.height), int(cam.width)
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        a = torch.empty((5, H, W), dtype=torch.float32, device=dev) if aux else None
        c = torch.empty((H, W), dtype=torch.int32, device=dev) if count else None
        opts = render_opts(use_mlp, rgb_residual, bg, flags)
        fn = mgs_render_checked if checked else mgs_render
        fn(self.ws, scene, cam, opts, rgb, a, c, stream)
        return {"rgb": rgb, "aux": a, "count": c}

    def render_depth(self, scene, cam, use_mlp=False, rgb_residual=False, flags=0, stream=None):
        """Colour and depth image (Eq. 5 depth), then a workspace sync."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        H, W = int(cam.height), int(cam.width)
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        depth = torch.empty((H, W), dtype=torch.float32, device=dev)
        opts = render_opts(use_mlp, rgb_residual, (0.0, 0.0, 0.0), flags)
        for attempt in range(2):
            mgs_render_depth(self.ws, scene, cam, opts, rgb, depth, stream)
            st, _ = mgs_workspace_sync(self.ws, stream, allow_overflow=True)
            if st == MGS_OK:
                break
        if st != MGS_OK:
            raise MGSError(st, "depth render overflowed its tile lists twice")
        return {"rgb": rgb, "depth": depth}

    def tile_lists(self, stream=None):
        """Copies of the last render's tile lists as numpy arrays (offsets, gids)."""
        torch = self.torch
        n, k = mgs_tile_lists(self.ws, stream=stream)
        dev = torch.device("cuda", self.device)
        off = torch.empty(n + 1, dtype=torch.int32, device=dev)
        gids = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
        mgs_tile_lists(self.ws, off, gids, stream=stream)
        return (off.cpu().numpy().view(np.uint32).astype(np.int64),
                gids[:k].cpu().numpy().view(np.uint32).astype(np.int64))

    def close(self):
        for s in self._scenes:
            mgs_unload_scene(s)
        self._scenes = []
        if self.ws is not None:
            mgs_workspace_destroy(self.ws)
            self.ws = None
        if self.ctx is not None:
            mgs_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
