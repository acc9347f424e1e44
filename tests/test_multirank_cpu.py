"""The benchmark's multi-GPU path on CPU: two gloo ranks.  Ranks own disjoint
clip seeds (no data-path collective), the only collective is the max of the
per-rank times, and the whole-job rate divides all ranks' audio by it."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [3.0, 5.0][rank]
    ms = bench.reduce_max(ms_local, "cpu")
    rate = bench.whole_job_rate(640.0, world, ms * 1e-3)
    out.put((rank, bench.shard_seed0(rank), ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, ms0, rate0), (r1, s1, ms1, rate1) = res
    assert ms0 == ms1 == 5.0                  # max over ranks
    assert rate0 == rate1 == 2 * 640.0 / 5e-3  # whole-job audio-s/s
    import bench
    assert abs(s1 - s0) >= bench.N_CLIPS      # disjoint seed ranges
