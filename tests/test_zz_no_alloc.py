"""cwth_execute_direct_noalloc: the direct path for callers that cannot
allocate device memory while they run (their memory belongs to another
allocator, a real-time loop must not stall on cudaMalloc/cudaFree, or the
process must not grow after start-up).  Its scratch is a fixed array inside
libcwth.so.

The tests call the entry point through the C ABI several times in a row,
with different batches, scale lists and hops (so each call runs on scratch
the previous one left behind), and check each result

  * byte for byte against the planned direct path (cwth_plan + cwth_execute
    run the same kernels on identically built tables), including a request
    of more than 128 scales, which takes two GEMM groups;
  * against the float64 oracle, within the tolerances the parity tests use;

and that a bounded wait that runs out is reported once by
cwth_noalloc_status and then cleared.  This file is named to be collected
last.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16": 2e-2, "bf16x2": 1e-5, "bf16x3": 1e-5}


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
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.cwth_execute_direct_noalloc(
        ctypes.byref(w), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), S, hop,
        cw.PREC[precision], ctypes.c_void_p(xs.data_ptr()), int(xs.stride(0)), int(xs.shape[1]),
        ctypes.c_void_p(lengths.data_ptr() if lengths is not None else 0), int(xs.shape[0]),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert st == 0, (st, lib.cwth_last_error())
    assert lib.cwth_noalloc_status(ctypes.c_void_p(stream)) == 0
    return out.cpu().numpy()


def test_noalloc_matches_planned_direct_path_and_oracle(cw):
    import oracle
    from paper_2408_14302_gb300 import signals
    cases = [
        # (clips, samples, scales, hop, precision, lengths)
        (3, 16000, signals.scales_for_band(100, 8000, 40, 16000.0), 64, "bf16x2", None),
        (5, 9000, signals.scales_for_band(150, 6000, 24, 16000.0), 128, "bf16",
         [9000, 8999, 1, 0, 4097]),
        (2, 10000, signals.scales_for_band(100, 8000, 32, 16000.0), 256, "bf16x3", [10000, 5003]),
        # 200 scales: two GEMM groups (128 + 72), each with its own bank
        # slot, schedule slot and tensor maps inside the scratch array
        (2, 12000, signals.scales_for_band(100, 8000, 200, 16000.0), 64, "bf16x2", [12000, 7001]),
    ]
    for clips, n, scales, hop, precision, lengths in cases:
        xs = np.stack([signals.machine_clip(300 + i, n) for i in range(clips)])
        xd = torch.from_numpy(np.ascontiguousarray(xs, np.float32)).cuda()
        ld = torch.tensor(lengths, dtype=torch.int64, device="cuda") if lengths else None
        got = _noalloc(cw, xd, scales, hop, precision, ld)
        ref = _planned(cw, xd, scales, hop, precision, ld)
        assert got.shape == ref.shape
        # Same kernels on identically built tables: identical bytes,
        # including the untouched frames past each clip.
        assert np.array_equal(got, ref), (precision, hop, len(scales))
        for i in range(clips):
            L = n if lengths is None else lengths[i]
            F = -(-L // hop)
            assert np.all(got[i, :, F:] == -5.0), "frames past the clip were written"
            if L == 0:
                continue
            want = oracle.cwth_magnitude(xs[i, :L].astype(np.float32).astype(np.float64),
                                         scales, hop)
            err = float(np.max(np.abs(got[i, :, :F] - want))) / float(want.max())
            assert err <= TOL[precision], (precision, i, err)


def test_noalloc_timeout_is_reported_once_then_cleared(cw):
    """A bounded wait that runs out (forced by the self-test on the
    allocation-free status word: a wait of 10^6 cycles on a barrier nothing
    arrives on) is reported by the next status check, once; afterwards the
    entry point works again."""
    from paper_2408_14302_gb300 import signals
    lib = cw.lib()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.cwth_noalloc_status(ctypes.c_void_p(stream)) == 0
    assert lib.cwth_selftest_wait_timeout(None, 1_000_000, ctypes.c_void_p(stream)) == 0
    assert lib.cwth_noalloc_status(ctypes.c_void_p(stream)) == 5  # CWTH_ERR_TIMEOUT
    assert lib.cwth_noalloc_status(ctypes.c_void_p(stream)) == 0
    n, hop = 8000, 64
    xs = np.stack([signals.machine_clip(77 + i, n) for i in range(2)])
    xd = torch.from_numpy(np.ascontiguousarray(xs, np.float32)).cuda()
    scales = signals.scales_for_band(200, 8000, 16, 16000.0)
    got = _noalloc(cw, xd, scales, hop, "bf16x2", None)
    ref = _planned(cw, xd, scales, hop, "bf16x2", None)
    assert np.array_equal(got, ref)


def test_noalloc_python_wrapper(cw):
    """The binding's wrapper runs the entry point and checks its own
    arguments before calling it."""
    from paper_2408_14302_gb300 import signals
    n, hop = 6000, 64
    scales = signals.scales_for_band(300, 8000, 12, 16000.0)
    xd = torch.from_numpy(signals.machine_batch(2, n)).cuda()
    out = torch.empty((2, 12, cw.num_frames(n, hop)), device="cuda")
    cw.execute_direct_noalloc(scales, hop, xd, out, precision="bf16x2")
    cw.noalloc_status()
    ref = _planned(cw, xd, scales, hop, "bf16x2", None)
    assert np.array_equal(out.cpu().numpy(), ref)
    with pytest.raises(ValueError):
        cw.execute_direct_noalloc(scales, hop, xd, out[:, :5])           # wrong shape
    with pytest.raises(ValueError):
        cw.execute_direct_noalloc(scales, hop, xd.double(), out)         # not float32
    with pytest.raises(ValueError):
        cw.execute_direct_noalloc(scales, hop, xd, out,
                                  lengths=torch.tensor([n, n], dtype=torch.int32, device="cuda"))


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
