"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: CPU only)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(mgs_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2603_11531_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    assert {"mgs_render", "mgs_load_scene", "mgs_workspace_sync"} <= names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b(mgs_\w+)$", out, flags=re.M))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_lists_every_declared_symbol():
    import paper_2603_11531_gb300 as m
    assert set(m.EXPORTS) == _declared()


def test_library_loads_without_gpu(built):
    import paper_2603_11531_gb300 as m
    L = m.lib()
    for name in m.EXPORTS:
        assert hasattr(L, name)
    assert "sm_103a" in m.mgs_version()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2603_11531_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="missing"):
        m.lib()


def test_no_cpu_fallback_in_package():
    """The renderer package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2603_11531_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path


def test_binding_rejects_bad_output_buffers_before_any_call(monkeypatch):
    """A wrong output buffer (host memory, wrong shape, dtype or layout) is a
    ValueError raised by the binding before the library is called, so the
    kernels never write through it."""
    import numpy as np
    import torch

    import paper_2603_11531_gb300 as m
    from paper_2603_11531_gb300 import synth

    def no_call():
        raise AssertionError("the library must not be called")

    monkeypatch.setattr(m, "lib", no_call)
    ws, scene = object(), object()
    monkeypatch.setitem(m._ws_dev, id(ws), 0)
    monkeypatch.setitem(m._scene_info, id(scene), (0, 100))
    ws_h, sc_h = id(ws), id(scene)
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 32, 24, 60.0)
    opts = m.render_opts()
    bad = [torch.empty((24, 32, 3)),                      # host memory
           np.empty((24, 32, 3), np.float32),             # numpy (host)
           None]
    for out in bad:
        with pytest.raises(ValueError):
            m.mgs_render(ws_h, sc_h, cam, opts, out)
        with pytest.raises(ValueError):
            m.mgs_render_checked(ws_h, sc_h, cam, opts, out)
    with pytest.raises(ValueError):
        m.mgs_render_depth(ws_h, sc_h, cam, opts, torch.empty((24, 32, 3)), None)
    for host in (np.empty((24, 32), np.float32), np.empty((24, 32, 3), np.float64),
                 torch.empty((24, 32, 3), dtype=torch.float16),
                 torch.empty((32, 24, 3)).transpose(0, 1)):
        with pytest.raises(ValueError):
            m.mgs_render_to_host(ws_h, sc_h, cam, opts, host)
    with pytest.raises(ValueError):
        m.mgs_render_backward(ws_h, sc_h, cam, opts, torch.empty((24, 32, 3)),
                              torch.empty((5, 24, 32)), torch.empty((100, 24)))
    with pytest.raises(ValueError):          # handle this module never created
        m.mgs_render(object(), sc_h, cam, opts, torch.empty((24, 32, 3)))


def test_camera_checks_run_before_any_device_work(built):
    """A camera with znear <= 0 (the projection divides by the view depth)
    or a non-finite pose is refused by the host-side check that every entry
    point shares, before any CUDA call (so it is testable without a GPU)."""
    import ctypes
    import math

    import paper_2603_11531_gb300 as m
    from paper_2603_11531_gb300 import synth
    L = m.lib()
    good = m.camera_struct(synth.look_at((0, 0, -3), (0, 0, 0), 64, 48, 60.0))
    fake_out = ctypes.c_void_p(256)     # never dereferenced: the check fails first
    for field, value in (("znear", 0.0), ("znear", -1.0), ("znear", math.inf), ("fx", math.nan)):
        cam = m.mgs_camera.from_buffer_copy(good)
        setattr(cam, field, value)
        st = L.mgs_render_static(None, 0, m.MGS_PREC_FP32, ctypes.byref(cam),
                                 ctypes.byref(m.render_opts()), fake_out, None)
        assert st == m.MGS_ERR_INVALID_ARG, (field, value)
    cam = m.mgs_camera.from_buffer_copy(good)
    cam.t[1] = math.inf
    st = L.mgs_render_static(None, 0, m.MGS_PREC_FP32, ctypes.byref(cam),
                             ctypes.byref(m.render_opts()), fake_out, None)
    assert st == m.MGS_ERR_INVALID_ARG
