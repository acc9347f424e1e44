"""Stored expected scalograms (tests/golden/*.json, written from the float64
oracle by tests/golden/make_golden.py): the oracle must keep reproducing
them (CPU), and the CUDA path must match them within the float32 tolerance
without running the oracle (GPU)."""
from __future__ import annotations

import glob
import hashlib
import json
import os

import numpy as np
import pytest

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json")))
TOL_FP32 = 1e-5


def load(path):
    with open(path) as f:
        doc = json.load(f)
    from paper_2408_14302_gb300 import signals
    inp = doc["input"]
    assert inp["generator"] == "signals.tones_clip"
    x = np.ascontiguousarray(signals.tones_clip(inp["seed"], inp["samples"], inp["fs"]),
                             np.float32)
    return doc, x, np.asarray(doc["scales"]), np.asarray(doc["magnitude"])


def test_golden_files_present():
    assert len(GOLDEN) >= 3


@pytest.mark.parametrize("path", GOLDEN, ids=lambda p: os.path.basename(p)[:-5])
def test_oracle_reproduces_golden(path):
    import oracle
    doc, x, sc, mag = load(path)
    assert hashlib.sha1(x.tobytes()).hexdigest() == doc["input"]["sha1"]
    got = oracle.cwth_magnitude(x.astype(np.float64), sc, doc["hop"],
                                bandwidth=doc["morlet"]["bandwidth"],
                                center=doc["morlet"]["center"])
    assert got.shape == mag.shape
    assert np.max(np.abs(got - mag)) <= 1e-12 * np.max(mag)


@pytest.mark.gpu
@pytest.mark.parametrize("path", GOLDEN, ids=lambda p: os.path.basename(p)[:-5])
def test_gpu_matches_golden(path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth
    doc, x, sc, mag = load(path)
    with cwth.Plan(sc, hop=doc["hop"], max_len=len(x), bandwidth=doc["morlet"]["bandwidth"],
                   center=doc["morlet"]["center"]) as plan:
        out = plan.execute(torch.from_numpy(x[None]).cuda())
        torch.cuda.synchronize()
        got = out.cpu().numpy()[0].astype(np.float64)
    assert got.shape == mag.shape
    assert np.max(np.abs(got - mag)) <= TOL_FP32 * np.max(mag)
