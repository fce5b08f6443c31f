"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry
point include/*.h declares, and validates its arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2011_05427_gb300 import build, trt
    build.build()
    return trt.lib()


def declared_symbols():
    out = set()
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            src = open(os.path.join(ROOT, "include", name)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            out |= set(re.findall(r"\b(trt_[a-z0-9_]+)\s*\(", src))
    return sorted(out)


def test_every_declared_symbol_is_exported(L):
    from paper_2011_05427_gb300 import trt
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(trt.EXPORTED)


def _args(trt, nx=10, N=4, G=8, levels=(8, 1), precision=0, edges=None):
    e = np.ascontiguousarray(edges if edges is not None else
                             np.concatenate([[0.0], np.logspace(-3, 1, G - 1), [np.inf]]))
    lv = np.ascontiguousarray(levels, np.int32)
    keep = (e, lv)
    grid = trt.trt_grid(nx, None, 1.0, 1.0, 0.0)
    ang = trt.trt_angles(N)
    grp = trt.trt_groups(G, e.ctypes.data_as(trt._dp), 0.0, 0.0, lv.size,
                         lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    opt = trt.trt_options(precision, 1e-3, None, None, 0)
    return grid, ang, grp, opt, keep


def test_workspace_bytes_and_validation(L):
    from paper_2011_05427_gb300 import trt
    grid, ang, grp, opt, keep = _args(trt)
    n64 = L.trt_workspace_bytes(ctypes.byref(grid), ctypes.byref(ang), ctypes.byref(grp),
                                ctypes.byref(opt))
    assert n64 > 0 and n64 % 256 == 0
    opt.precision = 1
    n32 = L.trt_workspace_bytes(ctypes.byref(grid), ctypes.byref(ang), ctypes.byref(grp),
                                ctypes.byref(opt))
    assert 0 < n32 < n64          # FP32 intensity buffers in mixed mode
    # the pair low-order form adds the pair opacity tables, cell terms and row constants
    for base, n_base in ((trt.TRT_FP64, n64), (trt.TRT_SWEEP_FP32, n32)):
        opt.precision = base | trt.TRT_LO_PAIR
        npair = L.trt_workspace_bytes(ctypes.byref(grid), ctypes.byref(ang), ctypes.byref(grp),
                                      ctypes.byref(opt))
        assert npair > n_base and npair % 256 == 0
    # FP32 and pair group solves exclude each other; no other precision bits exist
    bad = [dict(nx=0), dict(N=0), dict(levels=(8, 3, 1)), dict(levels=(8, 2)),
           dict(levels=(4, 1)), dict(precision=7), dict(precision=6), dict(precision=8),
           dict(precision=-1),
           dict(edges=np.array([0.0, 1.0, 0.5, 2, 3, 4, 5, 6, np.inf]))]
    for kw in bad:
        g2, a2, gr2, o2, keep2 = _args(trt, **kw)
        assert L.trt_workspace_bytes(ctypes.byref(g2), ctypes.byref(a2), ctypes.byref(gr2),
                                     ctypes.byref(o2)) == 0, kw
        h = ctypes.c_void_p()
        op = trt.trt_opacity(1.0)
        rc = L.trt_create(ctypes.byref(g2), ctypes.byref(a2), ctypes.byref(gr2),
                          ctypes.byref(op), 0.008, ctypes.byref(o2), ctypes.byref(h))
        assert rc == trt.TRT_EINVAL and not h.value, kw
        assert L.trt_last_error(None)


def test_create_rejects_missing_workspace(L):
    from paper_2011_05427_gb300 import trt
    grid, ang, grp, opt, keep = _args(trt)
    h = ctypes.c_void_p()
    op = trt.trt_opacity(1.0)
    rc = L.trt_create(ctypes.byref(grid), ctypes.byref(ang), ctypes.byref(grp), ctypes.byref(op),
                      0.008, ctypes.byref(opt), ctypes.byref(h))
    assert rc == trt.TRT_EINVAL and not h.value
    assert b"workspace" in L.trt_last_error(None)
    assert L.trt_step(None, 1e-3, None, None) == trt.TRT_EINVAL
    assert L.trt_destroy(None) == trt.TRT_OK


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2011_05427_gb300 import trt
    monkeypatch.setattr(trt, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(trt, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        trt.lib()
