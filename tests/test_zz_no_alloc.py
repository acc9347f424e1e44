"""cwth_execute_direct_noalloc: the direct path for callers that cannot
allocate device memory while they run (their memory belongs to another
allocator, or cudaMalloc would stall a real-time or captured loop).  Its
scratch is a fixed array inside libcwth.so.

The test calls the entry point through the C ABI twice in a row, with
different batches, scale lists and hops (so the second call runs on scratch
the first one left behind), and checks each result against the planned
direct path (cwth_plan + cwth_execute) within the tolerances the parity
tests use.  This file is named to be collected last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16": 2e-2, "bf16x2": 1e-5}


@pytest.fixture(scope="module")
def cw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth
    return cwth


def _planned(cw, xs, scales, hop, precision, lengths):
    with cw.Plan(scales, hop=hop, max_len=xs.shape[1], precision=precision, path="direct") as p:
        out = torch.full((xs.shape[0], len(scales), p.frames_max), -5.0, device="cuda")
        p.execute(xs, lengths=lengths, out=out)
        p.sync()
        return out.cpu().numpy()


def _noalloc(cw, xs, scales, hop, precision, lengths):
    S = len(scales)
    F = cw.num_frames(xs.shape[1], hop)
    out = torch.full((xs.shape[0], S, F), -5.0, device="cuda")
    lib = cw.lib()
    sc = np.ascontiguousarray(np.asarray(scales, np.float64))
    w = cw.Morlet(1.5, 1.0)
    st = lib.cwth_execute_direct_noalloc(
        ctypes.byref(w), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), S, hop,
        cw.PREC[precision], ctypes.c_void_p(xs.data_ptr()), int(xs.stride(0)), int(xs.shape[1]),
        ctypes.c_void_p(lengths.data_ptr() if lengths is not None else 0), int(xs.shape[0]),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, (st, lib.cwth_last_error())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_planned_direct_path_twice(cw):
    from paper_2408_14302_gb300 import signals
    cases = [
        # (clips, samples, scales, hop, precision, lengths)
        (3, 16000, signals.scales_for_band(100, 8000, 40, 16000.0), 64, "bf16x2", None),
        (5, 9000, signals.scales_for_band(150, 6000, 24, 16000.0), 128, "bf16",
         [9000, 8999, 1, 0, 4097]),
    ]
    for clips, n, scales, hop, precision, lengths in cases:
        xs = np.stack([signals.machine_clip(300 + i, n) for i in range(clips)])
        xd = torch.from_numpy(np.ascontiguousarray(xs, np.float32)).cuda()
        ld = torch.tensor(lengths, dtype=torch.int64, device="cuda") if lengths else None
        got = _noalloc(cw, xd, scales, hop, precision, ld)
        ref = _planned(cw, xd, scales, hop, precision, ld)
        assert got.shape == ref.shape
        for i in range(clips):
            L = n if lengths is None else lengths[i]
            F = -(-L // hop)
            assert np.all(got[i, :, F:] == -5.0), "frames past the clip were written"
            if L == 0:
                continue
            scale = max(float(np.abs(ref[i, :, :F]).max()), 1e-30)
            err = float(np.max(np.abs(got[i, :, :F] - ref[i, :, :F]))) / scale
            assert err <= TOL[precision], (precision, i, err)


def test_noalloc_rejects_requests_beyond_its_scratch(cw):
    lib = cw.lib()
    sc = np.ascontiguousarray([2.0, 10.0], np.float64)
    w = cw.Morlet(1.5, 1.0)
    # 4096 clips of 160000 samples need ~2.6 GB of staged signal: refused
    # before anything runs (the pointers are never dereferenced).
    st = lib.cwth_execute_direct_noalloc(
        ctypes.byref(w), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, 64,
        cw.PREC["bf16"], ctypes.c_void_p(16), 160000, 160000, None, 4096, ctypes.c_void_p(16),
        None)
    assert st == 1
    assert b"bytes of scratch" in lib.cwth_last_error()
