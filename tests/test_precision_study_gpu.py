"""Precision study: tones generator, 1 s at 16 kHz, 128 scales 100-8000 Hz,
hops 64/128/256/512.  Each variant's max and RMS relative error against the
float64 oracle (max|err|/max|W| and rms(err)/rms(W) over the clip) must meet
its tolerance; the figures are written to precision_study.json in the
directory named by the CWTH_RESULTS_DIR environment variable, if set."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = [("direct", "bf16", 2e-2), ("direct", "bf16x2", 1e-5), ("direct", "bf16x3", 1e-5),
            ("direct", "fp32", 1e-5), ("spectral", "fp32", 1e-5)]


def test_precision_study():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2408_14302_gb300 import cwth, signals
    x = signals.tones_clip(seed=0, n=16000).astype(np.float32)
    sc = signals.scales_for_band(100, 8000, 128, 16000.0)
    xd = torch.from_numpy(x).cuda().unsqueeze(0)
    report = {}
    for hop in (64, 128, 256, 512):
        ref = oracle.cwth_magnitude(x.astype(np.float64), sc, hop)
        for path, prec, tol in VARIANTS:
            with cwth.Plan(sc, hop=hop, max_len=x.shape[0], precision=prec, path=path) as p:
                got = p.execute(xd)[0].cpu().numpy().astype(np.float64)
                p.sync()
            err = got - ref
            mx = float(np.max(np.abs(err)) / np.max(ref))
            rms = float(np.sqrt(np.mean(err ** 2)) / np.sqrt(np.mean(ref ** 2)))
            report[f"hop{hop}_{path}_{prec}"] = {"max_rel": mx, "rms_rel": rms, "tol": tol}
            assert mx <= tol, (hop, path, prec, mx)
    out = os.environ.get("CWTH_RESULTS_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_study.json"), "w") as f:
            json.dump(report, f, indent=1)
