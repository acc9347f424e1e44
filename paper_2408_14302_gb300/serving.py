"""Continuous-batching server for hop-size CWT requests.

Requests (one clip each, with its own length, scale count and hop) arrive
over time.  The scheduler admits them while a device-memory budget allows,
groups waiting requests that share (sample rate, scale count, hop) into
batches of up to `max_batch` clips, and keeps up to `max_inflight` batches on
the GPU at once, each on its own CUDA stream, so new arrivals start while
earlier work is still running.  Plans (with their float64-generated device
tables) are cached per (stream slot, rate, scales, hop, length bucket, path,
precision); a plan whose direct path owns staging memory is never shared by
two batches in flight.  Latency = completion time observed by the host -
arrival time.

`GpuExecutor` runs batches through libcwth.so (pinned host staging, async
copies, one event per batch); `MockExecutor` models durations on the CPU so
the admission and batching logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass

import numpy as np

from . import signals

GiB = 1 << 30


@dataclass
class Request:
    rid: int
    x: np.ndarray          # float32 samples
    n_scales: int
    hop: int
    fs: float = 16000.0
    arrival: float = 0.0   # seconds after the start of the run
    src: int = -1          # pool signal the clip was cut from (-1: none)
    start: int = 0         # first sample of the clip in that signal

    @property
    def key(self):
        return (float(self.fs), int(self.n_scales), int(self.hop))

    @property
    def frames(self) -> int:
        return -(-len(self.x) // self.hop)

    @property
    def audio_seconds(self) -> float:
        return len(self.x) / self.fs


@dataclass
class Result:
    rid: int
    out: np.ndarray | None
    arrival: float
    done: float
    batch_size: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def length_bucket(n: int, floor: int = 1 << 14) -> int:
    return max(floor, 1 << int(math.ceil(math.log2(max(n, 1)))))


def batch_bytes(reqs, direct: bool) -> int:
    """Device bytes a batch holds: padded input, output, staging."""
    L = length_bucket(max(len(r.x) for r in reqs))
    F = -(-L // min(r.hop for r in reqs))
    S = max(r.n_scales for r in reqs)
    b = len(reqs)
    return 4 * b * L + 4 * b * S * F + (8 * b * L if direct else 0)


class MockExecutor:
    """CPU stand-in: a batch takes `base_s + per_audio_s * audio seconds`."""

    def __init__(self, base_s: float = 1e-3, per_audio_s: float = 1e-4, direct: bool = False):
        self.base_s, self.per_audio_s, self.direct = base_s, per_audio_s, direct
        self.launched = []

    def cost(self, reqs) -> int:
        return batch_bytes(reqs, self.direct)

    def launch(self, reqs, slot: int):
        dur = self.base_s + self.per_audio_s * sum(r.audio_seconds for r in reqs)
        h = {"t_end": time.perf_counter() + dur, "reqs": reqs, "slot": slot}
        self.launched.append(h)
        return h

    def done(self, h) -> bool:
        return time.perf_counter() >= h["t_end"]

    def results(self, h):
        return [np.zeros((r.n_scales, r.frames), np.float32) for r in h["reqs"]]


class GpuExecutor:
    """Runs batches through libcwth.so.  form: "batched" uses the automatic
    path at `precision`; "per_clip" is the plain float32 spectral path."""

    def __init__(self, slots: int = 4, precision: str = "bf16x3", path: str = "auto",
                 f_lo: float = 50.0, f_hi: float = 8000.0, device: str = "cuda"):
        import torch
        from . import cwth
        self.torch, self.cwth = torch, cwth
        self.device = torch.device(device)
        self.precision, self.path = precision, path
        self.f_lo, self.f_hi = f_lo, f_hi
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.plans = {}
        self.bufs = {}
        self.direct = precision != "fp32" or path == "direct"

    def cost(self, reqs) -> int:
        return batch_bytes(reqs, self.direct)

    def _plan(self, slot, fs, S, hop, L):
        key = (slot, fs, S, hop, L, self.path, self.precision)
        p = self.plans.get(key)
        if p is None:
            scales = signals.scales_for_band(self.f_lo, min(self.f_hi, fs / 2.0), S, fs)
            p = self.cwth.Plan(scales, hop=hop, max_len=L, sample_rate=fs,
                               precision=self.precision, path=self.path)
            self.plans[key] = p
        return p

    def warm(self, fs_list, scale_counts, hops, lengths):
        """Build every plan the given request mix can need, for every stream
        slot, before serving (plans and their device tables stay cached)."""
        buckets = sorted({length_bucket(int(n)) for n in lengths})
        for slot in range(len(self.streams)):
            for fs in fs_list:
                for S in scale_counts:
                    for hop in hops:
                        for L in buckets:
                            self._plan(slot, float(fs), int(S), int(hop), L)

    def _buf(self, slot: int, name: str, numel: int, dtype, pinned: bool):
        """A slot's staging buffer of at least `numel` elements (grown on
        demand, reused by every batch the slot runs)."""
        torch = self.torch
        key = (slot, name)
        t = self.bufs.get(key)
        if t is None or t.numel() < numel:
            if pinned:
                t = torch.empty(numel, dtype=dtype).pin_memory()
            else:
                t = torch.empty(numel, dtype=dtype, device=self.device)
            self.bufs[key] = t
        return t[:numel]

    def launch(self, reqs, slot: int):
        """Copies the batch into the slot's pinned rows (only each clip's own
        samples: the kernels ignore samples past a clip's length, so no row is
        cleared), uploads, transforms and downloads on the slot's stream.
        A slot runs one batch at a time, so its buffers are free again when
        the server hands the slot out."""
        torch = self.torch
        fs, S, hop = reqs[0].key
        L = length_bucket(max(len(r.x) for r in reqs))
        plan = self._plan(slot, fs, S, hop, L)
        b = len(reqs)
        F = plan.frames_max
        hx = self._buf(slot, "hx", b * L, torch.float32, True).view(b, L)
        hl = self._buf(slot, "hl", b, torch.int64, True)
        hxn, hln = hx.numpy(), hl.numpy()
        for i, r in enumerate(reqs):
            hxn[i, : len(r.x)] = r.x
            hln[i] = len(r.x)
        xd = self._buf(slot, "xd", b * L, torch.float32, False).view(b, L)
        ld = self._buf(slot, "ld", b, torch.int64, False)
        od = self._buf(slot, "od", b * S * F, torch.float32, False).view(b, S, F)
        ho = self._buf(slot, "ho", b * S * F, torch.float32, True).view(b, S, F)
        st = self.streams[slot]
        with torch.cuda.stream(st):
            xd.copy_(hx, non_blocking=True)
            ld.copy_(hl, non_blocking=True)
            plan.execute(xd, lengths=ld, out=od, stream=st)
            ho.copy_(od, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"ev": ev, "reqs": reqs, "ho": ho, "slot": slot}

    def done(self, h) -> bool:
        return h["ev"].query()

    def results(self, h):
        ho = h["ho"].numpy()
        return [ho[i, :, : r.frames].copy() for i, r in enumerate(h["reqs"])]

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans.clear()
        self.bufs.clear()


class Server:
    """Open-loop replay of timed requests with continuous batching."""

    def __init__(self, executor, budget_bytes: int = 40 * GiB, max_batch: int = 16,
                 max_inflight: int = 4, batched: bool = True, keep_outputs: bool = True):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.max_batch = max_batch if batched else 1
        self.max_inflight = max_inflight
        self.keep_outputs = keep_outputs
        self.peak_bytes = 0
        self.rejected = []

    def _take_batch(self, pending):
        """The oldest waiting request plus later ones with the same key and
        length bucket (a batch is padded to its longest clip, so mixing
        lengths would transform padding)."""
        first = pending.popleft()
        batch = [first]
        if self.max_batch > 1:
            want = (first.key, length_bucket(len(first.x)))
            rest = collections.deque()
            while pending and len(batch) < self.max_batch:
                r = pending.popleft()
                (batch if (r.key, length_bucket(len(r.x))) == want else rest).append(r)
            while rest:
                pending.appendleft(rest.pop())
        return batch

    def run(self, requests, poll_s: float = 2e-4):
        reqs = sorted(requests, key=lambda r: r.arrival)
        n = len(reqs)
        pending = collections.deque()
        inflight = []          # (handle, bytes)
        free_slots = list(range(self.max_inflight))
        used = 0
        results = []
        nxt = 0
        t0 = time.perf_counter()
        while len(results) + len(self.rejected) < n:
            now = time.perf_counter() - t0
            while nxt < n and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # completions
            still = []
            for h, nbytes in inflight:
                if self.ex.done(h):
                    t_done = time.perf_counter() - t0
                    outs = self.ex.results(h) if self.keep_outputs else [None] * len(h["reqs"])
                    for r, o in zip(h["reqs"], outs):
                        results.append(Result(r.rid, o, r.arrival, t_done, len(h["reqs"])))
                    used -= nbytes
                    free_slots.append(h["slot"])
                else:
                    still.append((h, nbytes))
            inflight = still
            # admissions: launch while a stream slot and budget are free
            launched = False
            while pending and free_slots:
                batch = self._take_batch(pending)
                nbytes = self.ex.cost(batch)
                while nbytes > self.budget - used and len(batch) > 1:
                    pending.appendleft(batch.pop())      # shrink to fit
                    nbytes = self.ex.cost(batch)
                if nbytes > self.budget:
                    self.rejected.extend(batch)          # can never fit
                    continue
                if nbytes > self.budget - used:
                    for r in reversed(batch):
                        pending.appendleft(r)            # wait for memory
                    break
                slot = free_slots.pop()
                h = self.ex.launch(batch, slot)
                used += nbytes
                self.peak_bytes = max(self.peak_bytes, used)
                inflight.append((h, nbytes))
                launched = True
            if not launched:
                if nxt < n and not inflight and not pending:
                    time.sleep(max(0.0, min(reqs[nxt].arrival - (time.perf_counter() - t0),
                                            0.01)))
                else:
                    time.sleep(poll_s)
        wall = time.perf_counter() - t0
        return results, wall


def poisson_requests(n: int, rate: float, seed: int = 5000, pool=None, pool_seconds: float = 60.0,
                     fs: float = 16000.0, min_s: float = 0.5, max_s: float = 60.0,
                     scale_counts=(32, 64, 128, 256), hops=(32, 64, 128, 256, 512)):
    """Exponential inter-arrivals at `rate` per second; clip lengths log-
    uniform in [min_s, max_s]; scale count and hop uniform over the sets.
    Clips are cut from a pool of seeded machine-sound signals."""
    rng = np.random.default_rng(seed)
    if pool is None:
        pool = [signals.machine_clip(seed + i, int(pool_seconds * fs), fs) for i in range(8)]
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        secs = math.exp(rng.uniform(math.log(min_s), math.log(max_s)))
        L = max(1, int(round(secs * fs)))
        k = int(rng.integers(len(pool)))
        src = pool[k]
        start = int(rng.integers(0, max(1, len(src) - L)))
        x = np.ascontiguousarray(src[start:start + L], np.float32)
        out.append(Request(i, x, int(rng.choice(scale_counts)), int(rng.choice(hops)), fs, t,
                           k, start))
    return out


def summarize(results, wall):
    lat = np.array([r.latency for r in results]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean([r.batch_size for r in results])),
            "completed": len(results), "wall_s": wall}


def prepare_mix(server, fs=16000.0, scale_counts=(32, 64, 128, 256), hops=(32, 64, 128, 256, 512),
                min_s=0.5, max_s=60.0):
    """Builds the server's plans for every (scales, hop, length bucket) key
    that poisson_requests with these parameters can produce."""
    lo, hi = length_bucket(int(min_s * fs)), length_bucket(int(max_s * fs))
    buckets = []
    b = lo
    while b <= hi:
        buckets.append(b)
        b *= 2
    for S in scale_counts:
        for hop in hops:
            for b in buckets:
                server.prepare(fs, S, hop, b)


def library_replay(reqs, pinned_pool, out_ring, budget_bytes=40 * GiB, plan_cache_bytes=4 * GiB,
                   max_batch=16, slots=4, precision="fp32", path="auto", dry_run=False,
                   server=None):
    """Replays `reqs` through the library's server (cwth_server_replay: the
    admission loop, batching, copies and launches all in C).  Each request's
    samples are read in place from `pinned_pool` (a page-locked torch tensor
    [signals, samples] holding the pool the clips were cut from) and its
    scalogram written into `out_ring` (a page-locked float32 tensor used as
    a ring: outputs of long-finished requests are overwritten).  Returns
    (summary dict, latencies in s, batch sizes).  dry_run: the server's
    dry-run mode (no device work; any CPU tensors will do).  server: an
    open cwth.Server to replay through (its plan cache carries over from
    earlier replays); otherwise one is made from the other arguments and
    closed afterwards."""
    from . import cwth
    n = len(reqs)
    arr = (cwth.Request * n)()
    base = pinned_pool.data_ptr()
    row = pinned_pool.shape[1]
    ring = out_ring.data_ptr()
    cap = out_ring.numel()
    off = 0
    for i, q in enumerate(reqs):
        if q.src < 0:
            raise ValueError("library_replay needs requests cut from the pool (src >= 0)")
        m = q.n_scales * q.frames
        if off + m > cap:
            off = 0
        arr[i] = cwth.Request(q.rid, base + 4 * (q.src * row + q.start), len(q.x), q.fs,
                              q.n_scales, q.hop, ring + 4 * off)
        off += m
    srv = server or cwth.Server(budget_bytes=budget_bytes, plan_cache_bytes=plan_cache_bytes,
                                max_batch=max_batch, slots=slots, precision=precision, path=path,
                                dry_run=dry_run)
    try:
        before = srv.stats()
        lat, bs, stat, wall = srv.replay(arr, np.array([q.arrival for q in reqs]))
        st = srv.stats()
    finally:
        if server is None:
            srv.close()
    if np.any(stat != 0):
        raise RuntimeError(f"{int(np.sum(stat != 0))} requests failed: {sorted(set(stat.tolist()))}")
    lat_ms = lat * 1e3
    return ({"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
             "mean_batch": float(np.mean(bs)),
             "completed": int(st["completed"] - before["completed"]), "wall_s": wall,
             "peak_gb": st["peak_bytes"] / GiB, "plans": st["plans"],
             "evictions": int(st["evictions"] - before["evictions"]),
             "rejected": int(st["rejected"] - before["rejected"])}, lat, bs)


def main(argv=None):
    """Sweep arrival rates through the library's server (default) or the
    Python scheduler:
    python -m paper_2408_14302_gb300.serving --rates 50,200,1000,2000 --requests 400"""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="50,100,200,500,1000,2000")
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--plan-cache-gb", type=float, default=16.0)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--engine", default="library", choices=["library", "python"])
    ap.add_argument("--forms", default="batched_auto_fp32,batched_auto_bf16x3,"
                    "per_clip_fp32_spectral")
    a = ap.parse_args(argv)
    import torch
    pool = [signals.machine_clip(5000 + i, 60 * 16000, 16000.0) for i in range(8)]
    forms = {"batched_auto_fp32": dict(precision="fp32", path="auto", batched=True),
             "batched_spectral_fp32": dict(precision="fp32", path="spectral", batched=True),
             "batched_auto_bf16x3": dict(precision="bf16x3", path="auto", batched=True),
             "per_clip_fp32_spectral": dict(precision="fp32", path="spectral", batched=False)}
    forms = {k: forms[k] for k in a.forms.split(",")}
    if a.engine == "library":
        pinned = torch.from_numpy(np.stack(pool).astype(np.float32)).pin_memory()
        ring = torch.empty(1 << 29, dtype=torch.float32).pin_memory()   # 2 GiB of outputs
    for name, f in forms.items():
        mb = a.max_batch if f["batched"] else 1
        if a.engine == "library":
            from . import cwth
            srv = cwth.Server(budget_bytes=int(a.budget_gb * GiB),
                              plan_cache_bytes=int(a.plan_cache_gb * GiB), max_batch=mb,
                              slots=a.slots, precision=f["precision"], path=f["path"])
            # warm: the server's plans for every key of the mix (shared
            # float32 plans: 4 scale counts x 5 hops x 7 length buckets; they
            # stay cached), then one pass of back-to-back requests
            if f["precision"] == "fp32":
                prepare_mix(srv)
            warm = poisson_requests(min(1000, a.requests), 1e6, seed=4000, pool=pool)
            library_replay(warm, pinned, ring, server=srv)
            for rate in [float(r) for r in a.rates.split(",")]:
                reqs = poisson_requests(a.requests, rate, seed=5000 + int(rate), pool=pool)
                torch.cuda.synchronize()
                s, _, _ = library_replay(reqs, pinned, ring, server=srv)
                audio = sum(r.audio_seconds for r in reqs)
                s.update({"engine": "library", "form": name, "rate_req_s": rate,
                          "audio_sec_per_s": audio / s["wall_s"],
                          "offered_audio_sec_per_s": audio / reqs[-1].arrival})
                print(json.dumps(s), flush=True)
            srv.close()
            continue
        ex = GpuExecutor(slots=a.slots, precision=f["precision"], path=f["path"])
        ex.warm([16000.0], (32, 64, 128, 256), (32, 64, 128, 256, 512),
                [0.5 * 16000, 60 * 16000] + [2 ** k for k in range(14, 21)])
        # warm the kernels with one pass of back-to-back requests
        warm = poisson_requests(min(60, a.requests), 1e6, seed=4000, pool=pool)
        Server(ex, int(a.budget_gb * GiB), a.max_batch, a.slots, f["batched"],
               keep_outputs=False).run(warm)
        for rate in [float(r) for r in a.rates.split(",")]:
            reqs = poisson_requests(a.requests, rate, seed=5000 + int(rate), pool=pool)
            srv = Server(ex, int(a.budget_gb * GiB), a.max_batch, a.slots, f["batched"],
                         keep_outputs=False)
            torch.cuda.synchronize()
            res, wall = srv.run(reqs)
            s = summarize(res, wall)
            audio = sum(r.audio_seconds for r in reqs)
            s.update({"engine": "python", "form": name, "rate_req_s": rate,
                      "audio_sec_per_s": audio / wall,
                      "offered_audio_sec_per_s": audio / reqs[-1].arrival,
                      "peak_gb": srv.peak_bytes / GiB, "rejected": len(srv.rejected)})
            print(json.dumps(s), flush=True)
        ex.close()


if __name__ == "__main__":
    main()
