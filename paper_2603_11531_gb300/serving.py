"""Python binding of the continuous-batching render server (mgs_server_*).

Argument marshalling only; admission, graphs, batching and completion all run
in the library (a worker thread inside libmobilegs.so).
"""
from __future__ import annotations

import ctypes

from . import (MGS_ERR_TIMEOUT, MGSError, _check, _check_dev_tensor, _ctx_dev, _dev_of, _ptr,
               camera_struct, lib, mgs_camera)

_sig_done = False


class mgs_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64)]


def _L():
    global _sig_done
    L = lib()
    if not _sig_done:
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        L.mgs_server_create.argtypes = [P, ctypes.POINTER(mgs_server_config), PP]
        L.mgs_server_create.restype = I32
        L.mgs_server_destroy.argtypes = [P]
        L.mgs_server_destroy.restype = I32
        L.mgs_server_submit.argtypes = [P, P, ctypes.POINTER(mgs_camera), P, P,
                                        ctypes.POINTER(I64)]
        L.mgs_server_submit.restype = I32
        L.mgs_server_wait.argtypes = [P, I64, D]
        L.mgs_server_wait.restype = I32
        L.mgs_server_ticket.argtypes = [P, I64, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                        ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]
        L.mgs_server_ticket.restype = I32
        L.mgs_server_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                       ctypes.POINTER(I64), ctypes.POINTER(I64),
                                       ctypes.POINTER(I32)]
        L.mgs_server_stats.restype = I32
        L.mgs_now.argtypes = []
        L.mgs_now.restype = D
        _sig_done = True
    return L


def mgs_now() -> float:
    return _L().mgs_now()


class Server:
    """Continuous-batching server over resident scenes of one context."""

    def __init__(self, ctx, slots: int = 8, max_batch: int = 8, hbm_budget_bytes: int = 8 << 30):
        cfg = mgs_server_config(slots, max_batch, hbm_budget_bytes)
        self.device = _dev_of(ctx, _ctx_dev, "context")
        h = ctypes.c_void_p()
        _check(_L().mgs_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h

    def submit(self, scene, cam, opts, out_rgb) -> int:
        """out_rgb: contiguous CUDA float32 tensor (H, W, 3) on the server's
        device; it must stay alive until the ticket completes."""
        import torch
        c = cam if isinstance(cam, mgs_camera) else camera_struct(cam)
        _check_dev_tensor(out_rgb, (int(c.height), int(c.width), 3), torch.float32, self.device,
                          "out_rgb")
        t = ctypes.c_int64()
        _check(_L().mgs_server_submit(self.h, scene, ctypes.byref(c), ctypes.byref(opts),
                                      _ptr(out_rgb), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: float = 60000.0, allow_timeout=False) -> int:
        st = _L().mgs_server_wait(self.h, int(ticket), float(timeout_ms))
        if st == MGS_ERR_TIMEOUT and allow_timeout:
            return st
        _check(st)
        return st

    def ticket(self, ticket: int) -> dict:
        s, r = ctypes.c_int32(), ctypes.c_int32()
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(_L().mgs_server_ticket(self.h, int(ticket), ctypes.byref(s), ctypes.byref(r),
                                      ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"state": s.value, "result": r.value, "t_submit": a.value, "t_admit": b.value,
                "t_done": c.value}

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        g = ctypes.c_int32()
        _check(_L().mgs_server_stats(self.h, *[ctypes.byref(x) for x in v], ctypes.byref(g)))
        return {"completed": v[0].value, "queued": v[1].value, "running": v[2].value,
                "workspace_bytes": v[3].value, "graphs": bool(g.value)}

    def close(self):
        if getattr(self, "h", None) is not None:
            _check(_L().mgs_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Server", "mgs_now", "MGSError"]
