"""Host logic of uneven-length batching: grouping keys, length buckets, the
persisted autotuning cache and the workload recipe."""
from __future__ import annotations

import json

from paper_2408_14302_gb300 import batching


def test_length_bucket_and_keys():
    assert batching.length_bucket(1) == 1
    assert batching.length_bucket(16000) == 16384
    assert batching.length_bucket(16384) == 16384
    assert batching.group_key(16000, 64, 256) == (16000.0, 64, 256)


def test_tune_cache_persists(tmp_path):
    p = tmp_path / "c.json"
    c = batching.TuneCache(str(p))
    c.put("gpu|16000|64|256|262144|fp32", {"path": "spectral", "precision": "fp32", "ms": 0.2})
    again = batching.TuneCache(str(p))
    assert again.get("gpu|16000|64|256|262144|fp32")["path"] == "spectral"
    assert json.loads(p.read_text())


def test_uneven_workload_recipe():
    clips, fs, ns, hs = batching.uneven_workload(n_clips=40, min_s=0.01, max_s=0.05, seed=5)
    assert len(clips) == len(fs) == len(ns) == len(hs) == 40
    assert set(fs) <= {16000.0, 48000.0}
    assert set(ns) <= {64, 128} and set(hs) <= {128, 256, 512}
    for c, f in zip(clips, fs):
        assert 0.01 * f - 1 <= len(c) <= 0.05 * f + 1
