"""Uneven-length batches in one launch: every clip matches the float64
oracle, and the same clip transformed alone gives the same result as in the
mix (within the float32 tolerance), in the work-list mode (one kernel
launch over a device work list of every group's items) and in the graph
mode (one CUDA graph of per-group executes)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", params=["worklist", "graph"])
def batch(tmp_path_factory, request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import batching
    clips, fs, ns, hs = batching.uneven_workload(n_clips=18, seed=77, min_s=0.05, max_s=1.2,
                                                 p48k=0.3, scale_counts=(6, 10),
                                                 hops=(128, 256))
    cache = batching.TuneCache(str(tmp_path_factory.mktemp("tune") / "cache.json"))
    runner = batching.BatchRunner(clips, fs, ns, hs, cache=cache, mode=request.param)
    assert (runner.batch is not None) == (request.param == "worklist")
    runner.capture()
    runner.replay()
    torch.cuda.synchronize()
    yield runner, clips, fs, ns, hs, cache
    runner.close()


def test_every_clip_matches_the_oracle(batch):
    import oracle
    from paper_2408_14302_gb300 import signals
    runner, clips, fs, ns, hs, _ = batch
    assert len(runner.groups) >= 3
    for i in range(len(clips)):
        got = runner.result(i).astype(np.float64)
        sc = signals.scales_for_band(50.0, 8000.0, ns[i], fs[i])
        ref = oracle.cwth_magnitude(np.asarray(clips[i], np.float32).astype(np.float64), sc, hs[i])
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= TOL * np.max(ref), i


def test_alone_equals_in_the_mix(batch):
    from paper_2408_14302_gb300 import cwth, signals
    runner, clips, fs, ns, hs, _ = batch
    for i in (0, 5, 11):
        gi, _ = runner.where[i]
        path, prec, seg, radix = runner.groups[gi]["choice"]
        sc = signals.scales_for_band(50.0, 8000.0, ns[i], fs[i])
        with cwth.Plan(sc, hop=hs[i], max_len=len(clips[i]), sample_rate=fs[i], path=path,
                       precision=prec, seg_len=seg) as p:
            if radix:
                p.set_inverse_radix(radix)
            alone = p.execute(torch.from_numpy(np.asarray(clips[i], np.float32)).cuda())[0]
            alone = alone.cpu().numpy()
        mixed = runner.result(i)
        assert np.max(np.abs(alone - mixed)) <= TOL * np.max(np.abs(alone))


def test_replay_is_repeatable_and_cache_is_written(batch):
    runner, _, _, _, _, cache = batch
    before = [runner.result(i).copy() for i in range(3)]
    runner.replay()
    torch.cuda.synchronize()
    for i in range(3):
        assert np.array_equal(before[i], runner.result(i))
    assert len(cache.data) == len(runner.groups)


def test_worklist_batch_matches_per_group_executes():
    """The work-list launch gives each group's cwth_execute result (byte for
    byte: the same kernel arithmetic per item), including clips of length 0
    and 1 and hops with an odd factor, and leaves frames past each clip
    untouched."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth, signals
    # hops 96 and 100: segments with an odd factor (column FFTs plus
    # radix-3/5 passes) in the same launch as power-of-two ones
    specs = [(16000.0, 12, 128, [9000, 1, 0, 4000]), (48000.0, 8, 256, [20000, 12345]),
             (16000.0, 20, 512, [30000]), (16000.0, 10, 96, [25000, 7777]),
             (16000.0, 6, 100, [18000])]
    groups, plans, refs = [], [], []
    for fs, S, hop, lens in specs:
        n = max(lens)
        xs = np.stack([signals.machine_clip(500 + i, n, fs) for i in range(len(lens))])
        sc = signals.scales_for_band(50.0, 8000.0, S, fs)
        p = cwth.Plan(sc, hop=hop, max_len=n, sample_rate=fs)
        x = torch.from_numpy(xs.astype(np.float32)).cuda()
        ld = torch.tensor(lens, dtype=torch.int64, device="cuda")
        out = torch.full((len(lens), S, p.frames_max), -2.0, device="cuda")
        ref = torch.full_like(out, -2.0)
        p.execute(x, lengths=ld, out=ref)
        groups.append((p, x, ld, out, np.asarray(lens, np.int64)))
        plans.append(p)
        refs.append(ref)
    b = cwth.Batch(groups)
    assert b.items > 0
    for _ in range(2):  # the launch is repeatable
        b.execute()
        torch.cuda.synchronize()
        for (p, x, ld, out, lens), ref in zip(groups, refs):
            assert torch.equal(out, ref)
    b.close()
    for p in plans:
        p.close()


def test_worklist_mode_runs_pruned_groups_beside_the_launch():
    """Small hops give plans with pruned inverse FFTs, which the work list
    does not take: in the work-list mode those groups run as their own
    executes beside its launch (in the same graph), and every clip still
    matches the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2408_14302_gb300 import batching, signals
    clips, fs, ns, hs = batching.uneven_workload(n_clips=8, seed=91, min_s=0.05, max_s=0.8,
                                                 p48k=0.0, scale_counts=(6,), hops=(4, 128))
    runner = batching.BatchRunner(clips, fs, ns, hs, tune=False, mode="worklist")
    try:
        assert runner.solo and runner.batch is not None
        assert all(g["plan"].info()["spectral_pruned"] for g in runner.solo)
        runner.capture()
        runner.replay()
        torch.cuda.synchronize()
        for i in range(len(clips)):
            got = runner.result(i).astype(np.float64)
            sc = signals.scales_for_band(50.0, 8000.0, ns[i], fs[i])
            ref = oracle.cwth_magnitude(np.asarray(clips[i], np.float32).astype(np.float64), sc,
                                        hs[i])
            assert np.max(np.abs(got - ref)) <= TOL * np.max(ref), i
    finally:
        runner.close()
