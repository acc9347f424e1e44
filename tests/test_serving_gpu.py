"""The continuous-batching server on the GPU: every request's scalogram is
the same in the mix as alone (within 1e-5 of max|W|) and matches the float64
oracle within 1e-5 of max|W|, for the float32 form and the three-part split
bf16 form (whose per-product error, about 2^-24, holds on clips whose tap
products cancel)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,path", [("bf16x3", "auto"), ("fp32", "spectral")])
def test_mix_equals_alone_and_oracle(precision, path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2408_14302_gb300 import cwth, serving, signals
    pool = [signals.machine_clip(900 + i, 40000, 16000.0) for i in range(3)]
    reqs = serving.poisson_requests(30, 3000.0, seed=31, pool=pool, min_s=0.05, max_s=2.0,
                                    scale_counts=(8, 12), hops=(64, 128))
    ex = serving.GpuExecutor(slots=3, precision=precision, path=path)
    srv = serving.Server(ex, 1 << 34, max_batch=6, max_inflight=3, batched=True)
    res, _ = srv.run(reqs)
    ex.close()
    assert len(res) == len(reqs) and max(r.batch_size for r in res) > 1
    by_id = {r.rid: r for r in res}
    for q in reqs:
        got = by_id[q.rid].out
        sc = signals.scales_for_band(50.0, 8000.0, q.n_scales, q.fs)
        with cwth.Plan(sc, hop=q.hop, max_len=len(q.x), precision=precision, path=path) as p:
            alone = p.execute(torch.from_numpy(q.x).cuda())[0].cpu().numpy()
        assert got.shape == alone.shape
        assert np.max(np.abs(got - alone)) <= 1e-5 * np.max(alone), q.rid
        ref = oracle.cwth_magnitude(q.x.astype(np.float64), sc, q.hop)
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(ref), q.rid


@pytest.mark.parametrize("precision,path,pinned", [("bf16x3", "auto", False),
                                                  ("fp32", "auto", False),
                                                  ("fp32", "auto", True)])
def test_library_server_mix_equals_alone_and_oracle(precision, path, pinned):
    """The library's server (cwth_server_*): requests replayed at their
    arrival times in batches of one key give each request's scalogram as a
    plan of its own would (1e-5 of max|W|; the server derives the scales in
    C) and match the float64 oracle.  Pageable inputs take one upload per
    request; page-locked ones the batch's gather kernel."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2408_14302_gb300 import cwth, serving, signals
    pool = [signals.machine_clip(950 + i, 40000, 16000.0) for i in range(3)]
    # arrivals microseconds apart: requests wait together and share batches
    reqs = serving.poisson_requests(40, 1e6, seed=37, pool=pool, min_s=0.05, max_s=2.0,
                                    scale_counts=(8, 12), hops=(64, 96, 128))
    arr = (cwth.Request * len(reqs))()
    outs, keep = [], []
    for i, q in enumerate(reqs):
        if pinned:
            xt = torch.from_numpy(q.x).pin_memory()
            ot = torch.full((q.n_scales, q.frames), -1.0).pin_memory()
            keep += [xt, ot]
            xp, out, op = xt.data_ptr(), ot.numpy(), ot.data_ptr()
        else:
            out = np.full((q.n_scales, q.frames), -1.0, np.float32)
            xp, op = q.x.ctypes.data, out.ctypes.data
        outs.append(out)
        arr[i] = cwth.Request(q.rid, xp, len(q.x), q.fs, q.n_scales, q.hop, op)
    with cwth.Server(budget_bytes=1 << 34, plan_cache_bytes=1 << 30, max_batch=6, slots=3,
                     precision=precision, path=path) as srv:
        lat, bs, stat, wall = srv.replay(arr, [q.arrival for q in reqs])
        st = srv.stats()
    assert np.all(stat == 0) and st["completed"] == len(reqs) and bs.max() > 1
    assert np.all(lat >= 0)
    for q, got in zip(reqs, outs):
        sc = signals.scales_for_band(50.0, 8000.0, q.n_scales, q.fs)
        with cwth.Plan(sc, hop=q.hop, max_len=len(q.x), precision=precision, path=path) as p:
            alone = p.execute(torch.from_numpy(q.x).cuda())[0].cpu().numpy()
        assert np.max(np.abs(got - alone)) <= 1e-5 * np.max(alone), q.rid
        ref = oracle.cwth_magnitude(q.x.astype(np.float64), sc, q.hop)
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(ref), q.rid


def test_library_server_reports_a_plan_it_cannot_build():
    """A request whose plan the forced path cannot build (hop 11 on the
    spectral path) completes with that plan's status; the requests around
    it complete normally."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth, signals
    x = np.ascontiguousarray(signals.machine_clip(5, 8000), np.float32)
    specs = [(0, 64), (1, 11), (2, 128)]
    outs = [np.zeros((8, -(-len(x) // h)), np.float32) for _, h in specs]
    arr = (cwth.Request * 3)(*[cwth.Request(rid, x.ctypes.data, len(x), 16000.0, 8, h,
                                            o.ctypes.data) for (rid, h), o in zip(specs, outs)])
    with cwth.Server(budget_bytes=1 << 32, max_batch=4, slots=2, precision="fp32",
                     path="spectral") as srv:
        lat, bs, stat, wall = srv.replay(arr, [0.0, 0.0, 0.0])
    assert list(stat) == [0, 4, 0]
    assert outs[0].max() > 0 and outs[2].max() > 0 and outs[1].max() == 0
