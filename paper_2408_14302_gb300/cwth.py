"""Thin ctypes binding of libcwth.so (include/cwth.h).

Argument marshalling only: every step of the transform runs in the CUDA
library.  PyTorch provides device memory and the current stream.  There is
no CPU fallback: if the library is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcwth.so")

CWTH_OK = 0
STATUS = {0: "CWTH_OK", 1: "CWTH_ERR_INVALID_ARG", 2: "CWTH_ERR_OOM", 3: "CWTH_ERR_CUDA",
          4: "CWTH_ERR_UNSUPPORTED", 5: "CWTH_ERR_TIMEOUT", 6: "CWTH_ERR_BAD_PLAN"}
PREC = {"fp32": 0, "bf16": 1, "bf16x2": 2, "bf16x3": 3}
PATH = {"auto": 0, "spectral": 1, "direct": 2}

# Every symbol include/cwth.h declares.
EXPORTS = ("cwth_plan", "cwth_execute", "cwth_execute_host", "cwth_destroy",
           "cwth_num_frames", "cwth_status_string", "cwth_plan_query",
           "cwth_plan_scale_paths", "cwth_sync", "cwth_last_error",
           "cwth_execute_direct_noalloc", "cwth_plan_set_host_chunks",
           "cwth_selftest_wait_timeout", "cwth_measure_fp32_fma", "cwth_plan_resampled",
           "cwth_plan_segment", "cwth_noalloc_status", "cwth_batch_create",
           "cwth_batch_execute", "cwth_batch_items", "cwth_batch_destroy",
           "cwth_plan_reserve", "cwth_server_create", "cwth_server_submit", "cwth_server_poll",
           "cwth_server_stats_query", "cwth_server_plan_bytes", "cwth_server_replay",
           "cwth_server_destroy", "cwth_server_prepare", "cwth_plan_set_inverse_radix",
           "cwth_plan_stage_bytes", "cwth_plan_bind_stage")


class CwthError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.detail = detail
        msg = f"{where}: {STATUS.get(status, status)}"
        super().__init__(msg + (f" ({detail})" if detail else ""))


class Morlet(ctypes.Structure):
    _fields_ = [("bandwidth", ctypes.c_double), ("center_freq", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_double), ("plan_cache_bytes", ctypes.c_double),
                ("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("path", ctypes.c_int32),
                ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double), ("wavelet", Morlet),
                ("dry_run", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("rid", ctypes.c_int64), ("x", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("fs", ctypes.c_double), ("n_scales", ctypes.c_int32), ("hop", ctypes.c_int32),
                ("out", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    _fields_ = [("rid", ctypes.c_int64), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("bytes_in_use", ctypes.c_double), ("peak_bytes", ctypes.c_double),
                ("plan_bytes", ctypes.c_double), ("plans", ctypes.c_int32),
                ("evictions", ctypes.c_int32), ("launched_batches", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("pending", ctypes.c_int32), ("in_flight", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("num_scales", ctypes.c_int32), ("hop", ctypes.c_int32),
                ("max_len", ctypes.c_int64), ("frames_max", ctypes.c_int64),
                ("num_spectral", ctypes.c_int32), ("num_direct", ctypes.c_int32),
                ("seg_len", ctypes.c_int32), ("seg_frames", ctypes.c_int32),
                ("seg_halo", ctypes.c_int32), ("fold_len", ctypes.c_int32),
                ("num_segments", ctypes.c_int32), ("direct_taps", ctypes.c_int32),
                ("table_bytes", ctypes.c_int64), ("sample_rate", ctypes.c_double),
                ("resample", ctypes.c_int32), ("spectral_threads", ctypes.c_int32),
                ("spectral_pass_scales", ctypes.c_int32), ("spectral_pruned", ctypes.c_int32),
                ("num_fused", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("spectral_parts", ctypes.c_int32), ("inverse_radix", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libcwth.so not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.cwth_plan.argtypes = [ctypes.POINTER(Morlet), ctypes.POINTER(ctypes.c_double), i32, i32,
                              dp, i64, i32, i32, ctypes.POINTER(vp)]
    lib.cwth_plan.restype = ctypes.c_int
    lib.cwth_plan_resampled.argtypes = lib.cwth_plan.argtypes
    lib.cwth_plan_resampled.restype = ctypes.c_int
    lib.cwth_plan_segment.argtypes = lib.cwth_plan.argtypes[:8] + [i32, ctypes.POINTER(vp)]
    lib.cwth_plan_segment.restype = ctypes.c_int
    lib.cwth_execute.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    lib.cwth_execute.restype = ctypes.c_int
    lib.cwth_execute_host.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    lib.cwth_execute_host.restype = ctypes.c_int
    lib.cwth_plan_set_host_chunks.argtypes = [vp, i32]
    lib.cwth_plan_set_host_chunks.restype = ctypes.c_int
    lib.cwth_plan_set_inverse_radix.argtypes = [vp, i32]
    lib.cwth_plan_set_inverse_radix.restype = ctypes.c_int
    lib.cwth_plan_reserve.argtypes = [vp, i32, i64, i32]
    lib.cwth_plan_reserve.restype = ctypes.c_int
    lib.cwth_plan_stage_bytes.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_size_t)]
    lib.cwth_plan_stage_bytes.restype = ctypes.c_int
    lib.cwth_plan_bind_stage.argtypes = [vp, vp, ctypes.c_size_t]
    lib.cwth_plan_bind_stage.restype = ctypes.c_int
    lib.cwth_selftest_wait_timeout.argtypes = [vp, i64, vp]
    lib.cwth_selftest_wait_timeout.restype = ctypes.c_int
    lib.cwth_measure_fp32_fma.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    lib.cwth_measure_fp32_fma.restype = ctypes.c_int
    lib.cwth_destroy.argtypes = [vp]
    lib.cwth_destroy.restype = ctypes.c_int
    lib.cwth_num_frames.argtypes = [i64, i32]
    lib.cwth_num_frames.restype = i64
    lib.cwth_status_string.argtypes = [ctypes.c_int]
    lib.cwth_status_string.restype = ctypes.c_char_p
    lib.cwth_plan_query.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.cwth_plan_query.restype = ctypes.c_int
    lib.cwth_plan_scale_paths.argtypes = [vp, ctypes.POINTER(i32)]
    lib.cwth_plan_scale_paths.restype = ctypes.c_int
    lib.cwth_last_error.argtypes = []
    lib.cwth_last_error.restype = ctypes.c_char_p
    lib.cwth_sync.argtypes = [vp, vp]
    lib.cwth_sync.restype = ctypes.c_int
    lib.cwth_execute_direct_noalloc.argtypes = [ctypes.POINTER(Morlet),
                                                ctypes.POINTER(ctypes.c_double), i32, i32, i32,
                                                vp, i64, i64, vp, i32, vp, vp]
    lib.cwth_execute_direct_noalloc.restype = ctypes.c_int
    lib.cwth_noalloc_status.argtypes = [vp]
    lib.cwth_noalloc_status.restype = ctypes.c_int
    pp = ctypes.POINTER(vp)
    lib.cwth_batch_create.argtypes = [i32, pp, pp, ctypes.POINTER(i64), pp, pp,
                                      ctypes.POINTER(i32), pp, ctypes.POINTER(vp)]
    lib.cwth_batch_create.restype = ctypes.c_int
    lib.cwth_batch_execute.argtypes = [vp, vp]
    lib.cwth_batch_execute.restype = ctypes.c_int
    lib.cwth_batch_items.argtypes = [vp]
    lib.cwth_batch_items.restype = i64
    lib.cwth_batch_destroy.argtypes = [vp]
    lib.cwth_batch_destroy.restype = ctypes.c_int
    lib.cwth_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.cwth_server_create.restype = ctypes.c_int
    lib.cwth_server_submit.argtypes = [vp, ctypes.POINTER(Request), i32]
    lib.cwth_server_submit.restype = ctypes.c_int
    lib.cwth_server_poll.argtypes = [vp, ctypes.POINTER(Completion), i32]
    lib.cwth_server_poll.restype = ctypes.c_int32
    lib.cwth_server_stats_query.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.cwth_server_stats_query.restype = ctypes.c_int
    lib.cwth_server_plan_bytes.argtypes = [vp, dp, i32, i32, i64]
    lib.cwth_server_plan_bytes.restype = ctypes.c_double
    lib.cwth_server_replay.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_double),
                                       i32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.cwth_server_replay.restype = ctypes.c_int
    lib.cwth_server_prepare.argtypes = [vp, dp, i32, i32, i64]
    lib.cwth_server_prepare.restype = ctypes.c_int
    lib.cwth_server_destroy.argtypes = [vp]
    lib.cwth_server_destroy.restype = ctypes.c_int
    return lib


_lib = load_library()


def lib() -> ctypes.CDLL:
    return _lib


def _check(status: int, where: str):
    if status != CWTH_OK:
        detail = ""
        if status in (2, 3, 4):
            detail = (_lib.cwth_last_error() or b"").decode(errors="replace")
        raise CwthError(status, where, detail)


def measure_fp32_fma_tflops(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (cwth_measure_fp32_fma)."""
    v = ctypes.c_double()
    s = 0 if stream is None else stream.cuda_stream
    _check(_lib.cwth_measure_fp32_fma(ctypes.byref(v), ctypes.c_void_p(s)), "cwth_measure_fp32_fma")
    return v.value


def num_frames(n: int, hop: int) -> int:
    return int(_lib.cwth_num_frames(int(n), int(hop)))


def execute_direct_noalloc(scales, hop: int, x, out, lengths=None, precision: str = "bf16x2",
                           bandwidth: float = 1.5, center: float = 1.0, max_len=None,
                           stream=None):
    """cwth_execute_direct_noalloc: direct-path scalograms without any device
    allocation (scratch lives in a fixed array inside libcwth.so).  ``x``:
    float32 CUDA tensor [B, ld]; ``out``: float32 CUDA tensor
    [B, S, num_frames(max_len, hop)], written asynchronously."""
    import torch
    sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float64).ravel())
    if x.dim() == 1:
        x = x.unsqueeze(0)
    if x.dtype != torch.float32 or not x.is_cuda or x.stride(1) != 1:
        raise ValueError("x must be a float32 CUDA tensor with unit column stride")
    B = x.shape[0]
    max_len = int(x.shape[1]) if max_len is None else int(max_len)
    if lengths is not None and (lengths.dtype != torch.int64 or not lengths.is_cuda
                                or lengths.numel() != B or not lengths.is_contiguous()):
        raise ValueError("lengths must be a contiguous int64 CUDA tensor with one entry per clip")
    want = (B, int(sc.shape[0]), num_frames(max_len, hop))
    if (out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous()
            or tuple(out.shape) != want):
        raise ValueError(f"out must be a contiguous float32 CUDA tensor of shape {want}")
    ld = int(x.shape[1]) if B == 1 else int(x.stride(0))
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    w = Morlet(float(bandwidth), float(center))
    st = _lib.cwth_execute_direct_noalloc(
        ctypes.byref(w), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(sc.shape[0]),
        int(hop), PREC[precision], ctypes.c_void_p(x.data_ptr()), ld, max_len,
        ctypes.c_void_p(lengths.data_ptr() if lengths is not None else 0), int(B),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    _check(st, "cwth_execute_direct_noalloc")
    return out


def noalloc_status(stream=None):
    """cwth_noalloc_status: wait for ``stream`` and raise CwthError if an
    allocation-free call gave up a bounded wait since the last check (the
    status word is cleared by the check)."""
    s = 0 if stream is None else stream.cuda_stream
    _check(_lib.cwth_noalloc_status(ctypes.c_void_p(s)), "cwth_noalloc_status")


class Plan:
    """A cwth_plan_t: scales (in samples), hop, Morlet B/C and the longest clip.
    ``resample_first=True`` makes a cwth_plan_resampled plan (the signal is
    re-sampled at the hop spacing, then transformed at every sample with
    scales / hop); its inputs and output shape are the same.  ``seg_len`` > 0
    fixes the spectral path's FFT segment length (cwth_plan_segment)."""

    def __init__(self, scales, hop: int, max_len: int, bandwidth: float = 1.5,
                 center: float = 1.0, sample_rate: float = 16000.0,
                 precision: str = "fp32", path: str = "auto", resample_first: bool = False,
                 seg_len: int = 0):
        sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float64).ravel())
        self.scales = sc
        self.hop = int(hop)
        self.max_len = int(max_len)
        self.S = int(sc.shape[0])
        self._h = ctypes.c_void_p()
        w = Morlet(float(bandwidth), float(center))
        args = (ctypes.byref(w), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                self.S, self.hop, float(sample_rate), self.max_len, PREC[precision], PATH[path])
        if resample_first:
            if seg_len:
                raise ValueError("seg_len applies to cwth_plan_segment plans only")
            _check(_lib.cwth_plan_resampled(*args, ctypes.byref(self._h)), "cwth_plan_resampled")
        elif seg_len:
            _check(_lib.cwth_plan_segment(*args, int(seg_len), ctypes.byref(self._h)),
                   "cwth_plan_segment")
        else:
            _check(_lib.cwth_plan(*args, ctypes.byref(self._h)), "cwth_plan")
        self.frames_max = num_frames(self.max_len, self.hop)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        _check(_lib.cwth_plan_query(self._h, ctypes.byref(inf)), "cwth_plan_query")
        return inf.as_dict()

    def scale_paths(self) -> np.ndarray:
        out = np.zeros(self.S, np.int32)
        _check(_lib.cwth_plan_scale_paths(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "cwth_plan_scale_paths")
        return out

    def execute(self, x, lengths=None, out=None, stream=None):
        """Device batch ``x`` (torch float32 CUDA tensor [B, ld >= max_len]) ->
        ``out`` [B, S, frames_max] float32 on the same device."""
        import torch
        if x.dim() == 1:
            x = x.unsqueeze(0)
        if x.dtype != torch.float32 or not x.is_cuda or x.stride(1) != 1:
            raise ValueError("x must be a float32 CUDA tensor with unit column stride")
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, self.S, self.frames_max), dtype=torch.float32, device=x.device)
        if lengths is not None and (lengths.dtype != torch.int64 or not lengths.is_cuda):
            raise ValueError("lengths must be an int64 CUDA tensor")
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        # A single row's stride is meaningless (size-1 dims may carry any stride).
        ld = int(x.shape[1]) if B == 1 else int(x.stride(0))
        st = _lib.cwth_execute(self._h, ctypes.c_void_p(x.data_ptr()), ld,
                               ctypes.c_void_p(lengths.data_ptr() if lengths is not None else 0),
                               int(B), ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(stream.cuda_stream))
        _check(st, "cwth_execute")
        return out

    def execute_host(self, x, out, lengths=None, stream=None):
        """Host batch (numpy or pinned torch CPU tensor, float32 [B, ld]) ->
        host ``out`` [B, S, frames_max]; returns when ``out`` is filled."""
        def ptr(a):
            if a is None:
                return 0
            if hasattr(a, "data_ptr"):
                return a.data_ptr()
            return a.ctypes.data
        B = x.shape[0]
        if B == 1:
            ld = x.shape[1]
        else:
            ld = x.stride(0) if hasattr(x, "stride") and callable(x.stride) else x.strides[0] // 4
        s = 0
        if stream is not None:
            s = stream.cuda_stream
        st = _lib.cwth_execute_host(self._h, ctypes.c_void_p(ptr(x)), int(ld),
                                    ctypes.c_void_p(ptr(lengths)), int(B),
                                    ctypes.c_void_p(ptr(out)), ctypes.c_void_p(s))
        _check(st, "cwth_execute_host")
        return out

    def set_host_chunks(self, n: int):
        """Chunks of execute_host (0 = automatic); see cwth_plan_set_host_chunks."""
        _check(_lib.cwth_plan_set_host_chunks(self._h, int(n)), "cwth_plan_set_host_chunks")

    def set_inverse_radix(self, radix: int):
        """Inverse-FFT pass plan of the spectral path: 0 (cost model), 8 or
        16; see cwth_plan_set_inverse_radix."""
        _check(_lib.cwth_plan_set_inverse_radix(self._h, int(radix)),
               "cwth_plan_set_inverse_radix")

    def reserve(self, batch: int, ld_x: int = 0, host: bool = False):
        """Sizes the plan's growable workspaces for `batch` clips so later
        executes of at most that many clips allocate nothing; see
        cwth_plan_reserve."""
        _check(_lib.cwth_plan_reserve(self._h, int(batch), int(ld_x), 1 if host else 0),
               "cwth_plan_reserve")

    def stage_bytes(self, batch: int) -> int:
        """Bytes the direct path's staged bf16 signal needs for `batch`
        clips (0 without tensor-core scales); see cwth_plan_stage_bytes."""
        n = ctypes.c_size_t(0)
        _check(_lib.cwth_plan_stage_bytes(self._h, int(batch), ctypes.byref(n)),
               "cwth_plan_stage_bytes")
        return int(n.value)

    def bind_stage(self, buf=None):
        """Stage the direct path's signal in `buf` (a CUDA tensor the caller
        keeps alive, at least stage_bytes(batch) bytes) in later executes;
        None unbinds.  See cwth_plan_bind_stage."""
        if buf is None:
            _check(_lib.cwth_plan_bind_stage(self._h, None, 0), "cwth_plan_bind_stage")
            return
        if not buf.is_cuda or not buf.is_contiguous():
            raise ValueError("the staging buffer must be a contiguous CUDA tensor")
        _check(_lib.cwth_plan_bind_stage(self._h, ctypes.c_void_p(buf.data_ptr()),
                                         buf.numel() * buf.element_size()),
               "cwth_plan_bind_stage")

    def sync(self, stream=None):
        """Wait for this plan's work on ``stream`` and raise on device-side
        errors (a kernel that gave up a bounded wait)."""
        s = 0 if stream is None else stream.cuda_stream
        _check(_lib.cwth_sync(self._h, ctypes.c_void_p(s)), "cwth_sync")

    def close(self):
        if self._h:
            _check(_lib.cwth_destroy(self._h), "cwth_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """A cwth_batch_t: groups of (plan, device batch) run by one kernel launch.

    groups: list of (plan, x, lengths, out, host_lengths) with x a float32
    CUDA tensor [B, ld], lengths an int64 CUDA tensor [B] or None, out the
    float32 CUDA output [B, S, frames_max] and host_lengths a numpy int64
    array (or None).  The tensors must outlive the batch."""

    def __init__(self, groups):
        n = len(groups)
        vp = ctypes.c_void_p
        self._keep = []
        plans = (vp * n)(*[g[0].handle.value for g in groups])
        xs = (vp * n)(*[g[1].data_ptr() for g in groups])
        lds = (ctypes.c_int64 * n)(*[int(g[1].shape[1]) if g[1].shape[0] == 1
                                     else int(g[1].stride(0)) for g in groups])
        dl = (vp * n)(*[(g[2].data_ptr() if g[2] is not None else None) for g in groups])
        hl = []
        for g in groups:
            if g[4] is None:
                hl.append(None)
            else:
                a = np.ascontiguousarray(np.asarray(g[4], np.int64))
                self._keep.append(a)
                hl.append(a.ctypes.data)
        hla = (vp * n)(*hl)
        bs = (ctypes.c_int32 * n)(*[int(g[1].shape[0]) for g in groups])
        outs = (vp * n)(*[g[3].data_ptr() for g in groups])
        for g in groups:
            x, ln, out = g[1], g[2], g[3]
            if x.dtype.__str__() != "torch.float32" or not x.is_cuda or x.stride(1) != 1:
                raise ValueError("x must be a float32 CUDA tensor with unit column stride")
            if ln is not None and (str(ln.dtype) != "torch.int64" or not ln.is_cuda):
                raise ValueError("lengths must be an int64 CUDA tensor")
            if (str(out.dtype) != "torch.float32" or not out.is_cuda or not out.is_contiguous()
                    or tuple(out.shape) != (x.shape[0], g[0].S, g[0].frames_max)):
                raise ValueError("out must be a contiguous float32 CUDA tensor [B, S, frames_max]")
        self._h = vp()
        _check(_lib.cwth_batch_create(n, plans, xs, lds, dl, hla, bs, outs, ctypes.byref(self._h)),
               "cwth_batch_create")
        self.groups = groups

    @property
    def items(self) -> int:
        return int(_lib.cwth_batch_items(self._h))

    def execute(self, stream=None):
        """One kernel launch over every group, on ``stream`` (asynchronous)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(_lib.cwth_batch_execute(self._h, ctypes.c_void_p(stream.cuda_stream)),
               "cwth_batch_execute")

    def close(self):
        if self._h:
            _check(_lib.cwth_batch_destroy(self._h), "cwth_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Server:
    """The library's continuous-batching server (cwth_server_*): admission
    under a device-memory budget that includes cached plans, LRU plan cache,
    batches of one (rate, scales, hop, length bucket) key, per-slot streams,
    uploads from and downloads into the callers' buffers.  Requests are
    ``Request`` structs whose ``x`` / ``out`` point at host memory that stays
    valid until they complete (page-locked memory makes the copies DMA)."""

    def __init__(self, budget_bytes=40 << 30, plan_cache_bytes=4 << 30, max_batch=16, slots=4,
                 precision="fp32", path="auto", f_lo=50.0, f_hi=8000.0, bandwidth=1.5,
                 center=1.0, dry_run=False):
        cfg = ServerConfig(float(budget_bytes), float(plan_cache_bytes), int(max_batch), int(slots),
                           PREC[precision], PATH[path], float(f_lo), float(f_hi),
                           Morlet(float(bandwidth), float(center)), 1 if dry_run else 0)
        self._h = ctypes.c_void_p()
        _check(_lib.cwth_server_create(ctypes.byref(cfg), ctypes.byref(self._h)),
               "cwth_server_create")
        self._done = (Completion * 4096)()

    def submit(self, reqs):
        arr = reqs if isinstance(reqs, ctypes.Array) else (Request * len(reqs))(*reqs)
        _check(_lib.cwth_server_submit(self._h, arr, len(arr)), "cwth_server_submit")

    def poll(self):
        """[(rid, status, batch_size, t_done)] of the requests completed now."""
        k = _lib.cwth_server_poll(self._h, self._done, len(self._done))
        if k < 0:
            _check(-k, "cwth_server_poll")
        return [(c.rid, c.status, c.batch_size, c.t_done) for c in self._done[:k]]

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.cwth_server_stats_query(self._h, ctypes.byref(st)), "cwth_server_stats_query")
        return st.as_dict()

    def prepare(self, fs, n_scales, hop, n_max):
        """Builds the cached plan(s) requests of (fs, n_scales, hop) with up
        to n_max samples will use (cwth_server_prepare)."""
        _check(_lib.cwth_server_prepare(self._h, float(fs), int(n_scales), int(hop), int(n_max)),
               "cwth_server_prepare")

    def plan_bytes(self, fs, n_scales, hop, bucket) -> float:
        return _lib.cwth_server_plan_bytes(self._h, float(fs), int(n_scales), int(hop), int(bucket))

    def replay(self, reqs, arrival_s):
        """Open-loop replay (cwth_server_replay): returns (latency_s, batch
        sizes, statuses, wall seconds)."""
        import numpy as np
        arr = reqs if isinstance(reqs, ctypes.Array) else (Request * len(reqs))(*reqs)
        t = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(len(arr), np.float64)
        bs = np.zeros(len(arr), np.int32)
        stat = np.zeros(len(arr), np.int32)
        wall = ctypes.c_double()
        dptr = ctypes.POINTER(ctypes.c_double)
        _check(_lib.cwth_server_replay(self._h, arr, t.ctypes.data_as(dptr), len(arr),
                                       lat.ctypes.data_as(dptr),
                                       bs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       stat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       ctypes.byref(wall)), "cwth_server_replay")
        return lat, bs, stat, wall.value

    def close(self):
        if self._h:
            _check(_lib.cwth_server_destroy(self._h), "cwth_server_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
