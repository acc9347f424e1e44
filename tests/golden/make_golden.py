"""Writes the stored expected scalograms under tests/golden/.

Every value comes from the float64 oracle (``oracle.cwth_magnitude``: Eq. 1
of the paper, Sec. II.A, evaluated at b = k H, Sec. II.B) on seeded
synthetic inputs from ``paper_2408_14302_gb300.signals``; nothing here runs
the CUDA path.  The inputs are stored as their recipe plus the SHA-1 of the
float32 samples, so a change of the generator is detected.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2408_14302_gb300 import signals  # noqa: E402

CASES = [
    # name, seed, samples, f_lo, f_hi, scales, hop
    ("tones_4000_8scales_hop64", 11, 4000, 100.0, 8000.0, 8, 64),
    ("tones_256_4scales_hop1", 12, 256, 1000.0, 8000.0, 4, 1),
    ("tones_3000_6scales_hop256", 13, 3000, 50.0, 4000.0, 6, 256),
]
FS = 16000.0


def case_input(seed, n):
    return np.ascontiguousarray(signals.tones_clip(seed, n, FS), np.float32)


def main():
    for name, seed, n, f_lo, f_hi, S, hop in CASES:
        x = case_input(seed, n)
        sc = signals.scales_for_band(f_lo, f_hi, S, FS)
        mag = oracle.cwth_magnitude(x.astype(np.float64), sc, hop)
        doc = {
            "source": "oracle.cwth_magnitude (float64; Eq. 1 at b = k H, Sec. II.A-B), "
                      "written by tests/golden/make_golden.py",
            "input": {"generator": "signals.tones_clip", "seed": seed, "samples": n,
                      "fs": FS, "dtype": "float32",
                      "sha1": hashlib.sha1(x.tobytes()).hexdigest()},
            "morlet": {"bandwidth": 1.5, "center": 1.0},
            "band_hz": [f_lo, f_hi], "scales": [float(a) for a in sc], "hop": hop,
            "magnitude": [[float(v) for v in row] for row in mag],
        }
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(doc, f, indent=0)
            f.write("\n")
        print(name, mag.shape)


if __name__ == "__main__":
    main()
