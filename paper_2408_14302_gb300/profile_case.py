"""Run one hop-size CWT workload repeatedly, for profilers.

    python -m paper_2408_14302_gb300.profile_case --path direct --precision bf16 \
        --signal tones --clips 512 --seconds 1 --scales 128 --f-lo 100 --hop 64

Builds the plan, runs `--warmup` executes, then `--reps` timed executes and
prints the mean CUDA-event time per execute.  Inputs are the seeded
synthetic generators; nothing here checks results (the test-suite does).
"""
from __future__ import annotations

import argparse

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--path", default="spectral", choices=["auto", "spectral", "direct"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "bf16x2"])
    ap.add_argument("--signal", default="machine", choices=["machine", "tones"])
    ap.add_argument("--clips", type=int, default=64)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--fs", type=float, default=16000.0)
    ap.add_argument("--scales", type=int, default=64)
    ap.add_argument("--f-lo", type=float, default=50.0)
    ap.add_argument("--f-hi", type=float, default=8000.0)
    ap.add_argument("--hop", type=int, default=256)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)

    import torch

    from paper_2408_14302_gb300 import cwth, signals

    n = int(round(a.seconds * a.fs))
    distinct = min(a.clips, 64)
    if a.signal == "machine":
        base = np.stack([signals.machine_clip(1000 + i, n, a.fs) for i in range(distinct)])
    else:
        base = np.stack([signals.tones_clip(seed=i, n=n, fs=a.fs) for i in range(distinct)])
    xs = np.ascontiguousarray(np.resize(base.astype(np.float32), (a.clips, n)))
    scales = signals.scales_for_band(a.f_lo, a.f_hi, a.scales, a.fs)
    plan = cwth.Plan(scales, hop=a.hop, max_len=n, precision=a.precision, path=a.path,
                     sample_rate=a.fs)
    x = torch.from_numpy(xs).cuda()
    out = torch.empty((a.clips, a.scales, plan.frames_max), device="cuda")
    for _ in range(a.warmup):
        plan.execute(x, out=out)
    plan.sync()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(a.reps):
        plan.execute(x, out=out)
    t1.record()
    plan.sync()
    print(f"{a.path}/{a.precision} hop {a.hop} clips {a.clips}: "
          f"{t0.elapsed_time(t1) / max(a.reps, 1):.4f} ms per execute; plan {plan.info()}")


if __name__ == "__main__":
    main()
