"""Host-side checks of the C ABI: the library loads, exports every function
include/cwth.h declares, and rejects bad arguments before touching the GPU."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "cwth.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cwth_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def cw():
    from paper_2408_14302_gb300 import build
    build.build()
    from paper_2408_14302_gb300 import cwth
    return cwth


def test_header_compiles_as_plain_c(tmp_path):
    """The boundary is a C ABI: include/cwth.h must stand alone in C99
    (every type it names comes from a standard header it includes)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "cwth.h"\nint main(void) { return (int)sizeof(cwth_plan_info) == 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "use_header.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_header_declares_the_expected_entry_points():
    decl = _declared_functions()
    for name in ("cwth_plan", "cwth_execute", "cwth_destroy", "cwth_num_frames",
                 "cwth_status_string", "cwth_execute_host"):
        assert name in decl


def test_library_exports_every_declared_symbol(cw):
    lib = cw.lib()
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} missing from libcwth.so"
    assert set(cw.EXPORTS) <= set(_declared_functions())


def test_num_frames_and_status_strings(cw):
    lib = cw.lib()
    assert lib.cwth_num_frames(16000, 64) == 250
    assert lib.cwth_num_frames(16001, 64) == 251
    assert lib.cwth_num_frames(0, 64) == 0
    assert lib.cwth_num_frames(10, 0) == 0
    assert lib.cwth_status_string(0) == b"CWTH_OK"
    assert lib.cwth_status_string(4) == b"CWTH_ERR_UNSUPPORTED"
    assert lib.cwth_status_string(99) == b"CWTH_ERR_UNKNOWN"


def _plan_status(cw, scales, hop=64, max_len=1000, B=1.5, C=1.0, fs=16000.0, prec=0, path=0,
                 null_out=False, null_w=False, null_scales=False):
    lib = cw.lib()
    sc = np.ascontiguousarray(np.asarray(scales, np.float64))
    h = ctypes.c_void_p()
    w = cw.Morlet(B, C)
    st = lib.cwth_plan(None if null_w else ctypes.byref(w),
                       None if null_scales else sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       len(sc), hop, fs, max_len, prec, path, None if null_out else ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw", [
    dict(scales=[2.0], hop=0), dict(scales=[2.0], hop=-4), dict(scales=[2.0], max_len=0),
    dict(scales=[0.0]), dict(scales=[-1.0]), dict(scales=[float("nan")]),
    dict(scales=[float("inf")]), dict(scales=[2.0], B=0.0), dict(scales=[2.0], C=-1.0),
    dict(scales=[2.0], fs=0.0), dict(scales=[2.0], prec=7), dict(scales=[2.0], path=9),
    dict(scales=[2.0], null_out=True), dict(scales=[2.0], null_w=True),
    dict(scales=[2.0], null_scales=True),
])
def test_plan_rejects_bad_arguments(cw, kw):
    st, h = _plan_status(cw, **kw)
    assert st == 1
    assert not h.value


def test_empty_scale_list_rejected(cw):
    lib = cw.lib()
    h = ctypes.c_void_p()
    w = cw.Morlet(1.5, 1.0)
    sc = (ctypes.c_double * 1)(2.0)
    assert lib.cwth_plan(ctypes.byref(w), sc, 0, 64, 16000.0, 100, 0, 0, ctypes.byref(h)) == 1


def test_plan_segment_rejects_bad_segment_lengths(cw):
    # Argument checks run before any device call, so no GPU is needed.
    lib = cw.lib()
    h = ctypes.c_void_p()
    w = cw.Morlet(1.5, 1.0)
    sc = (ctypes.c_double * 1)(2.0)
    # 3000 = 2^3 * 375, 11264 = 2^10 * 11, 16896 = 2^9 * 33: odd parts the
    # forward FFT does not take
    for seg in (-1, 256, 3000, 11264, 16896, 65536):
        assert lib.cwth_plan_segment(ctypes.byref(w), sc, 1, 64, 16000.0, 100, 0, 0, seg,
                                     ctypes.byref(h)) == 1, seg
        assert not h.value


def test_null_plan_handles(cw):
    lib = cw.lib()
    assert lib.cwth_destroy(None) == 0
    assert lib.cwth_execute(None, None, 0, None, 0, None, None) == 6
    assert lib.cwth_execute_host(None, None, 0, None, 0, None, None) == 6
    assert lib.cwth_plan_set_host_chunks(None, 2) == 6
    assert lib.cwth_plan_reserve(None, 4, 0, 0) == 6
    assert lib.cwth_plan_set_inverse_radix(None, 8) == 6
    # (a NULL plan there names the allocation-free entry point's status
    # word, which needs a device; a budget out of range is refused first)
    assert lib.cwth_selftest_wait_timeout(None, 0, None) == 1
    info = cw.PlanInfo()
    assert lib.cwth_plan_query(None, ctypes.byref(info)) == 6
    assert lib.cwth_plan_scale_paths(None, None) == 6


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2408_14302_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "cwth_oracle" not in text, f


def test_noalloc_wrapper_checks_arguments_before_the_library(cw):
    """execute_direct_noalloc refuses host tensors, wrong dtypes and a
    mis-shaped output before anything reaches the C ABI (no GPU needed)."""
    torch = pytest.importorskip("torch")
    x = torch.zeros((2, 1000), dtype=torch.float32)
    out = torch.zeros((2, 3, 16), dtype=torch.float32)
    with pytest.raises(ValueError):
        cw.execute_direct_noalloc([2.0, 4.0, 8.0], 64, x, out)          # host memory
    with pytest.raises(ValueError):
        cw.execute_direct_noalloc([2.0, 4.0, 8.0], 64, x.double(), out)  # float64


def test_plan_wrappers_marshal_their_arguments(cw, monkeypatch):
    """The binding's plan methods that need no tensor pass their arguments
    through unchanged (checked against a stand-in library, no device)."""
    calls = []

    class Fake:
        def __getattr__(self, name):
            def f(*a):
                calls.append((name, a))
                return 0
            return f

    monkeypatch.setattr(cw, "_lib", Fake())
    p = object.__new__(cw.Plan)
    p._h = ctypes.c_void_p(12345)
    try:
        p.reserve(8, ld_x=100, host=True)
        p.reserve(3)
        p.set_host_chunks(2)
        p.close()
    finally:
        p._h = ctypes.c_void_p()
    assert [c[0] for c in calls] == ["cwth_plan_reserve", "cwth_plan_reserve",
                                     "cwth_plan_set_host_chunks", "cwth_destroy"]
    assert calls[0][1][1:] == (8, 100, 1) and calls[1][1][1:] == (3, 0, 0)
    assert calls[2][1][1:] == (2,)
