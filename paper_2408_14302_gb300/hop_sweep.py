"""Hop sweep: the cost of the hop-size CWT as a function of the hop H.

The paper's method computes the CWT only at positions spaced by the hop
(Sec. II.B) and sweeps the hop to trade cost against recognition accuracy
(Sec. III); this module measures the cost side of that curve on the GPU: one
batch of machine-sound clips, a fixed scale bank, and for every hop the time
of one cwth_execute on the float32 spectral path and, where the hop allows
the tensor-core direct path (H a multiple of 8), on the split-bf16 automatic
path (both within 1e-5 of max|W|).  With --resample it also times the
resample-first reading of the hop (Sec. III.B, Fig. 2: re-sample the signal
at spacing H, then transform every sample with scales a / H) beside the
output-decimation transform, both on the scales the re-sampled signal can
represent (centre frequencies up to fs / (2 H)).

    python -m paper_2408_14302_gb300.hop_sweep [--clips 64] [--seconds 10] [--scales 64]

Prints one JSON line per (hop, evaluation).  Timing: CUDA events on the
launching stream, L2 flushed (256 MiB write) before every timed execute.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import cwth, signals

FLUSH_BYTES = 256 << 20


def time_execute(torch, plan, x, out, stream, flush, reps):
    for _ in range(3):
        plan.execute(x, out=out, stream=stream)
    plan.sync(stream)
    times = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.execute(x, out=out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    plan.sync(stream)
    return statistics.median(times)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--clips", type=int, default=64)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--fs", type=float, default=16000.0)
    ap.add_argument("--scales", type=int, default=64)
    ap.add_argument("--f-lo", type=float, default=50.0)
    ap.add_argument("--f-hi", type=float, default=8000.0)
    ap.add_argument("--hops", default="1,2,4,8,16,32,64,128,256,512,1024")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--resample", action="store_true")
    a = ap.parse_args(argv)
    import torch

    n = int(round(a.seconds * a.fs))
    xs = signals.machine_batch(a.clips, n, a.fs)
    sc = signals.scales_for_band(a.f_lo, min(a.f_hi, a.fs / 2), a.scales, a.fs)
    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(xs, np.float32)).to(dev)
    # The flush and the timed execute share one stream, so the flush has
    # finished before the execute starts.
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    audio = a.clips * n / a.fs
    for hop in (int(h) for h in a.hops.split(",")):
        forms = [("spectral", "fp32")]
        if hop % 8 == 0:
            forms.append(("auto", "bf16x3"))
        for path, precision in forms:
            try:
                plan = cwth.Plan(sc, hop=hop, max_len=n, sample_rate=a.fs, precision=precision,
                                 path=path)
            except cwth.CwthError as e:
                print(json.dumps({"hop": hop, "path": path, "precision": precision,
                                  "unsupported": str(e)}), flush=True)
                continue
            out = torch.empty((a.clips, a.scales, plan.frames_max), device=dev)
            ms = time_execute(torch, plan, x, out, stream, flush, a.reps)
            info = plan.info()
            print(json.dumps({
                "hop": hop, "path": path, "precision": precision, "ms": ms,
                "ms_per_clip": ms / a.clips, "audio_sec_per_s": audio / (ms * 1e-3),
                "scalogram_gbs": out.numel() * 4 / (ms * 1e-3) / 1e9,
                "frames": plan.frames_max, "num_spectral": info["num_spectral"],
                "num_direct": info["num_direct"], "seg_len": info["seg_len"],
                "num_segments": info["num_segments"]}), flush=True)
            plan.close()
            del out
        if not a.resample:
            continue
        f_top = min(a.f_hi, a.fs / (2 * hop))
        if f_top <= a.f_lo:
            print(json.dumps({"hop": hop, "resample_first": "skipped: no scale below fs/(2H)"}),
                  flush=True)
            continue
        sc_r = signals.scales_for_band(a.f_lo, f_top, a.scales, a.fs)
        for first in (False, True):
            plan = cwth.Plan(sc_r, hop=hop, max_len=n, sample_rate=a.fs, precision="fp32",
                             path="spectral" if not first else "auto", resample_first=first)
            out = torch.empty((a.clips, a.scales, plan.frames_max), device=dev)
            ms = time_execute(torch, plan, x, out, stream, flush, a.reps)
            print(json.dumps({
                "hop": hop, "form": "resample_first" if first else "output_decimation",
                "f_hi_hz": f_top, "precision": "fp32", "ms": ms, "ms_per_clip": ms / a.clips,
                "audio_sec_per_s": audio / (ms * 1e-3), "frames": plan.frames_max}), flush=True)
            plan.close()
            del out


if __name__ == "__main__":
    main()
