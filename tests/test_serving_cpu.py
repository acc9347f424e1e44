"""Scheduler logic of the continuous-batching server on the CPU (mock
executor): admission stays within the memory budget, oversize requests are
refused, same-key requests share batches, and requests that arrive while
others run start before those finish."""
from __future__ import annotations

import numpy as np

from paper_2408_14302_gb300 import serving


def _reqs(n, rate, seed=1, lens=(800, 4000), keys=((16, 64), (8, 128))):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        S, hop = keys[int(rng.integers(len(keys)))]
        x = np.zeros(int(rng.integers(*lens)), np.float32)
        out.append(serving.Request(i, x, S, hop, 16000.0, t))
    return out


def test_all_complete_within_budget():
    reqs = _reqs(60, 2000.0)
    ex = serving.MockExecutor(base_s=2e-3, per_audio_s=5e-3)
    budget = 3 * serving.batch_bytes(reqs[:4], False)
    srv = serving.Server(ex, budget, max_batch=4, max_inflight=3)
    res, wall = srv.run(reqs)
    assert len(res) == 60 and not srv.rejected
    assert srv.peak_bytes <= budget
    assert {r.rid for r in res} == set(range(60))
    assert all(r.latency >= 0 for r in res)


def test_batches_share_a_key_and_overlap_in_time():
    reqs = _reqs(40, 5000.0)
    ex = serving.MockExecutor(base_s=5e-3, per_audio_s=1e-3)
    srv = serving.Server(ex, 1 << 40, max_batch=8, max_inflight=4)
    res, _ = srv.run(reqs)
    for h in ex.launched:
        assert len({r.key for r in h["reqs"]}) == 1
    assert max(len(h["reqs"]) for h in ex.launched) > 1
    ends = sorted(h["t_end"] for h in ex.launched)
    starts = sorted(h["t_end"] - (5e-3 + 1e-3 * sum(r.audio_seconds for r in h["reqs"]))
                    for h in ex.launched)
    # some batch started before an earlier-started one ended: work overlapped
    assert any(s < e for s, e in zip(starts[1:], ends[:-1]))


def test_request_larger_than_budget_is_refused():
    big = serving.Request(0, np.zeros(50000, np.float32), 64, 32, 16000.0, 0.0)
    small = serving.Request(1, np.zeros(1000, np.float32), 8, 64, 16000.0, 0.0)
    ex = serving.MockExecutor()
    budget = serving.batch_bytes([small], False) * 2
    srv = serving.Server(ex, budget, max_batch=4, max_inflight=2)
    res, _ = srv.run([big, small])
    assert [r.rid for r in res] == [1]
    assert [r.rid for r in srv.rejected] == [0]


def test_per_clip_form_runs_one_request_per_batch():
    reqs = _reqs(12, 3000.0)
    ex = serving.MockExecutor()
    serving.Server(ex, 1 << 40, max_batch=16, max_inflight=2, batched=False).run(reqs)
    assert all(len(h["reqs"]) == 1 for h in ex.launched)


def test_library_replay_marshals_pool_and_ring():
    """serving.library_replay points each request into the sample pool and
    the output ring and replays them through the library's server (its
    dry-run mode: no device work)."""
    torch = __import__("pytest").importorskip("torch")
    pool = [np.arange(30000, dtype=np.float32) + 1e5 * k for k in range(3)]
    reqs = serving.poisson_requests(50, 1e5, seed=9, pool=pool, min_s=0.01, max_s=1.0,
                                    scale_counts=(4, 8), hops=(64, 128))
    pooled = torch.from_numpy(np.stack(pool))
    ring = torch.zeros(1 << 16)
    s, lat, bs = serving.library_replay(reqs, pooled, ring, max_batch=4, slots=2, dry_run=True)
    assert s["completed"] == 50 and s["rejected"] == 0 and s["mean_batch"] >= 1
    assert np.all(lat >= 0)
    # requests carry where they were cut from
    for q in reqs:
        assert np.array_equal(pool[q.src][q.start:q.start + len(q.x)], q.x)
