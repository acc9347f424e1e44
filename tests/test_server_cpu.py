"""Admission logic of the library's continuous-batching server
(cwth_server_*) in dry-run mode, on the CPU: no device work, plans costed by
cwth_server_plan_bytes, every launched batch completes at the next poll.
Checks that the budget charges cached plans as well as staging, that the
plan cache evicts least recently used idle plans, that a request that can
never fit is refused with CWTH_ERR_OOM, and that the replay loop completes
every request, batching those that wait together."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

OOM = 2


@pytest.fixture(scope="module")
def cw():
    from paper_2408_14302_gb300 import cwth
    return cwth


def _batch_bytes(b, L, S, hop):
    F = -(-L // hop)
    return 4.0 * b * L + 8.0 * b + 4.0 * b * S * F


def _requests(cw, specs, keep):
    """specs: (rid, n, S, hop); keep holds the buffers alive."""
    arr = (cw.Request * len(specs))()
    for i, (rid, n, S, hop) in enumerate(specs):
        x = np.zeros(n, np.float32)
        out = np.zeros(S * (-(-n // hop)), np.float32)
        keep += [x, out]
        arr[i] = cw.Request(rid, x.ctypes.data, n, 16000.0, S, hop, out.ctypes.data)
    return arr


def _drain(srv, n, limit=10000):
    done = []
    for _ in range(limit):
        done += srv.poll()
        if len(done) >= n:
            break
    return done


def test_budget_charges_cached_plans(cw):
    keep = []
    L, S, hop = 1 << 14, 16, 64
    with cw.Server(budget_bytes=1e12, max_batch=8, slots=4, dry_run=True) as probe:
        pb = probe.plan_bytes(16000.0, S, hop, L)
    assert pb > 0
    bb = _batch_bytes(1, L, S, hop)
    # Room for the plan and two clips of staging: without the plan's bytes
    # eight clips (two slots of four) would fit.
    budget = pb + 2 * bb + 1.0
    with cw.Server(budget_bytes=budget, plan_cache_bytes=1e12, max_batch=4, slots=2,
                   dry_run=True) as srv:
        srv.submit(_requests(cw, [(i, 1000, S, hop) for i in range(10)], keep))
        done = _drain(srv, 10)
        st = srv.stats()
    assert sorted(d[0] for d in done) == list(range(10))
    assert all(d[1] == 0 for d in done)
    assert max(d[2] for d in done) == 2
    assert st["plan_bytes"] == pytest.approx(pb) and st["plans"] == 1
    assert pb + 2 * bb - 1 <= st["peak_bytes"] <= budget


def test_plan_cache_evicts_least_recently_used(cw):
    keep = []
    L = 1 << 14
    with cw.Server(budget_bytes=1e12, dry_run=True) as probe:
        pa = probe.plan_bytes(16000.0, 16, 64, L)
        pb = probe.plan_bytes(16000.0, 32, 64, L)
    with cw.Server(budget_bytes=1e12, plan_cache_bytes=max(pa, pb) * 1.5, max_batch=4, slots=1,
                   dry_run=True) as srv:
        # keys alternate, one request at a time: every new plan needs the
        # idle other one evicted
        done = []
        for spec in [(0, 900, 16, 64), (1, 900, 32, 64), (2, 900, 16, 64)]:
            srv.submit(_requests(cw, [spec], keep))
            done += _drain(srv, 1)
        st = srv.stats()
    assert len(done) == 3 and all(d[1] == 0 for d in done)
    assert st["evictions"] == 2 and st["plans"] == 1
    assert st["plan_bytes"] <= max(pa, pb) * 1.5


def test_budget_charges_the_bf16_staging_of_a_batch(cw):
    """With tensor-core scales a batch also stages its bf16 signal (in its
    slot's buffer): the admission budget charges it, so a budget with room
    for the plan and one clip's samples, lengths, scalograms and bf16x3
    staging launches one clip at a time, where the same budget without the
    staging charge would hold two clips."""
    keep = []
    L, S, hop = 1 << 14, 16, 64
    with cw.Server(budget_bytes=1e12, max_batch=8, slots=4, precision="bf16x3",
                   dry_run=True) as probe:
        pb = probe.plan_bytes(16000.0, S, hop, L)
    bb = _batch_bytes(1, L, S, hop)
    sb = 2.0 * 3 * (L + 8192)          # the dry-run estimate: three bf16 parts
    budget = pb + bb + sb + 1.0
    assert budget >= pb + 2 * bb        # two clips fit without the staging charge
    with cw.Server(budget_bytes=budget, plan_cache_bytes=1e12, max_batch=4, slots=2,
                   precision="bf16x3", dry_run=True) as srv:
        srv.submit(_requests(cw, [(i, 1000, S, hop) for i in range(6)], keep))
        done = _drain(srv, 6)
        st = srv.stats()
    assert sorted(d[0] for d in done) == list(range(6))
    assert all(d[1] == 0 for d in done)
    assert max(d[2] for d in done) == 1
    assert st["plans"] == 1
    assert st["peak_bytes"] <= budget


def test_request_that_never_fits_is_refused(cw):
    keep = []
    L, S, hop = 1 << 15, 64, 32
    with cw.Server(budget_bytes=1e12, dry_run=True) as probe:
        pb = probe.plan_bytes(16000.0, S, hop, L)
    budget = pb + 0.5 * _batch_bytes(1, L, S, hop)
    with cw.Server(budget_bytes=budget, max_batch=4, slots=2, dry_run=True) as srv:
        srv.submit(_requests(cw, [(7, 20000, S, hop), (8, 500, 4, 64)], keep))
        done = {d[0]: d for d in _drain(srv, 2)}
        st = srv.stats()
    assert done[7][1] == OOM and done[8][1] == 0
    assert st["rejected"] == 1


def test_batches_hold_one_key_and_replay_completes(cw):
    keep = []
    rng = np.random.default_rng(3)
    specs = []
    for i in range(200):
        S, hop = [(8, 64), (16, 128), (8, 128)][int(rng.integers(3))]
        specs.append((i, int(rng.integers(100, 40000)), S, hop))
    arr = _requests(cw, specs, keep)
    arrivals = np.cumsum(rng.exponential(1e-5, len(specs)))
    with cw.Server(budget_bytes=1e12, max_batch=8, slots=3, dry_run=True) as srv:
        lat, bs, stat, wall = srv.replay(arr, arrivals)
        st = srv.stats()
    assert st["completed"] == 200 and st["pending"] == 0 and st["in_flight"] == 0
    assert np.all(lat >= 0) and np.all(bs >= 1) and bs.max() > 1 and np.all(stat == 0)
    assert wall >= arrivals[-1]
    # requests that waited together shared batches
    assert st["launched_batches"] < 200


def test_server_rejects_bad_arguments(cw):
    lib = cw.lib()
    h = ctypes.c_void_p()
    cfg = cw.ServerConfig(0.0, 1.0, 4, 2, 0, 0, 50.0, 8000.0, cw.Morlet(1.5, 1.0), 1)
    assert lib.cwth_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg = cw.ServerConfig(1e9, 1e9, 0, 2, 0, 0, 50.0, 8000.0, cw.Morlet(1.5, 1.0), 1)
    assert lib.cwth_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    with cw.Server(dry_run=True) as srv:
        bad = (cw.Request * 1)(cw.Request(0, None, 10, 16000.0, 8, 64, None))
        assert lib.cwth_server_submit(srv._h, bad, 1) == 1
        assert srv.stats()["pending"] == 0


def test_prepare_builds_the_plan_a_request_will_use(cw):
    keep = []
    with cw.Server(budget_bytes=1e12, max_batch=4, slots=3, dry_run=True) as srv:
        srv.prepare(16000.0, 16, 64, 1000)
        st = srv.stats()
        assert st["plans"] == 1 and st["plan_bytes"] == pytest.approx(
            srv.plan_bytes(16000.0, 16, 64, 1 << 14))
        srv.submit(_requests(cw, [(0, 900, 16, 64), (1, 16000, 16, 64)], keep))
        assert len(_drain(srv, 2)) == 2
        assert srv.stats()["plans"] == 1   # same key and bucket: no new plan
    with cw.Server(budget_bytes=1e12, max_batch=4, slots=3, precision="bf16x3",
                   dry_run=True) as srv:
        srv.prepare(16000.0, 16, 64, 1000)
        # bf16 staging lives in each slot's buffer: one plan per key
        assert srv.stats()["plans"] == 1
    with cw.Server(dry_run=True) as srv:
        with pytest.raises(cw.CwthError):
            srv.prepare(16000.0, 0, 64, 1000)
