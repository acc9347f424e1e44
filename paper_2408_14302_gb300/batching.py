"""Uneven-length batches: many clips with different lengths, sample rates,
scale counts and hops in one launch.

Clips are grouped by (sample rate, scale count, hop); each group is one plan
whose clips are packed into one padded device batch with a lengths vector.
Two modes:

* "worklist" (the default for the float32 accuracy class): every group's
  plan is a float32 plan of the spectral kernel (with its short-support
  scales summed in the time domain), and all groups are bound into one
  cwth_batch: a device work list of (group, clip, segment) items, longest
  first, run by ONE kernel launch (one block per item).  Groups whose plans
  the work list cannot take (small hops, whose plans prune their inverse
  FFTs, or 1024-thread segments) run as their own executes beside it.  The
  autotuner picks each group's FFT segment length (the cost model's, half
  or twice it) and its inverse FFTs' pass plan (radix 16 or 8).
* "graph": each group runs as its own `cwth_execute` (any path and
  precision, e.g. the tensor-core split-bf16 path) and all groups' executes
  are captured in one CUDA graph.  Its autotuner also tries the automatic
  path at three-part split-bf16 precision (within 1e-5 of max|W|).

Choices persist in a JSON cache keyed by GPU, sample rate, scale count,
hop, length bucket, accuracy class and mode.

Python orchestration only: the transform runs in libcwth.so.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import cwth, signals

# Candidate (path, precision) pairs per accuracy class.
CANDIDATES = {
    "fp32": [("spectral", "fp32"), ("auto", "bf16x3")],
    "bf16": [("auto", "bf16"), ("spectral", "fp32")],
}
# Candidates of the work-list mode: float32 plans of the spectral kernel.
WORKLIST_CANDIDATES = [("auto", "fp32")]


def default_cache_path() -> str:
    return os.environ.get("CWTH_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cwth_tune.json"))


class TuneCache:
    """Persisted autotuning decisions: key -> {"path", "precision", "seg_len", "ms"}
    (seg_len 0: the plan's own segment length)."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self._lock = threading.Lock()
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key: str):
        return self.data.get(key)

    def put(self, key: str, value: dict):
        with self._lock:
            self.data[key] = value
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            tmp = f"{self.path}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def length_bucket(n: int) -> int:
    """Power-of-two bucket of a clip length (tuning key granularity)."""
    return 1 << max(0, int(math.ceil(math.log2(max(n, 1)))))


def group_key(fs: float, n_scales: int, hop: int):
    return (float(fs), int(n_scales), int(hop))


def _worklist_ok(plan) -> bool:
    """Whether cwth_batch_create takes the plan: spectral-path scales only
    (folded or fused) in one part, two CTAs per SM, no pruned inverse FFTs,
    no re-sampling."""
    i = plan.info()
    return (i["num_direct"] == i["num_fused"] and not i["spectral_pruned"]
            and i["spectral_threads"] in (0, 512) and i["resample"] == 1
            and i["spectral_parts"] <= 1)


class BatchRunner:
    """Plans, packs and runs a list of uneven clips.

    clips: list of 1-D float arrays; fs, n_scales, hops: per-clip sample rate,
    scale count and hop; scales span f_lo..f_hi Hz geometrically (a_s = C fs/f).
    accuracy: "fp32" (1e-5 of max|W|) or "bf16" (2e-2).
    """

    def __init__(self, clips, fs, n_scales, hops, f_lo: float = 50.0, f_hi: float = 8000.0,
                 bandwidth: float = 1.5, center: float = 1.0, accuracy: str = "fp32",
                 tune: bool = True, cache: TuneCache | None = None, device: str = "cuda",
                 mode: str | None = None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.n = len(clips)
        self.bandwidth, self.center = bandwidth, center
        self.accuracy = accuracy
        self.mode = mode or ("worklist" if accuracy == "fp32" else "graph")
        if self.mode not in ("worklist", "graph"):
            raise ValueError("mode must be 'worklist' or 'graph'")
        self.cache = cache if cache is not None else (TuneCache() if tune else None)
        self.groups = []
        by_key = {}
        for i in range(self.n):
            by_key.setdefault(group_key(fs[i], n_scales[i], hops[i]), []).append(i)
        self.where = [None] * self.n  # clip -> (group index, row)
        gpu = torch.cuda.get_device_name(self.device)
        for gi, (key, idx) in enumerate(sorted(by_key.items())):
            gfs, S, hop = key
            lens = np.array([len(clips[i]) for i in idx], np.int64)
            max_len = int(lens.max())
            host = np.zeros((len(idx), max_len), np.float32)
            for r, i in enumerate(idx):
                host[r, : lens[r]] = clips[i]
                self.where[i] = (gi, r)
            scales = signals.scales_for_band(f_lo, min(f_hi, gfs / 2.0), S, gfs, center)
            g = {"key": key, "idx": idx, "lens": lens, "max_len": max_len, "scales": scales,
                 "x": torch.from_numpy(host).to(self.device),
                 "len_d": torch.from_numpy(lens).to(self.device)}
            g["choice"] = self._choose(g, gpu)
            g["plan"] = self._plan(g, *g["choice"])
            g["out"] = torch.zeros((len(idx), S, g["plan"].frames_max), device=self.device)
            self.groups.append(g)
        self.graph = None
        self.stream = torch.cuda.Stream(self.device)
        self.batch = None
        self.solo = list(self.groups)
        if self.mode == "worklist":
            # Groups whose plans the work list takes run in its one launch;
            # the others (pruned inverse FFTs, 1024-thread segments, direct
            # scales) keep their own executes beside it.
            wl = [g for g in self.groups if _worklist_ok(g["plan"])]
            self.solo = [g for g in self.groups if not _worklist_ok(g["plan"])]
            if wl:
                self.batch = cwth.Batch([(g["plan"], g["x"], g["len_d"], g["out"], g["lens"])
                                         for g in wl])

    # ------------------------------------------------------------ planning
    def _plan(self, g, path, precision, seg_len=0, radix=0):
        gfs, S, hop = g["key"]
        p = cwth.Plan(g["scales"], hop=hop, max_len=g["max_len"], bandwidth=self.bandwidth,
                      center=self.center, sample_rate=gfs, precision=precision, path=path,
                      seg_len=seg_len)
        if radix:
            p.set_inverse_radix(radix)
        return p

    def _choose(self, g, gpu):
        """(path, precision, seg_len, inverse radix) of the group: cached,
        else the fastest candidate; the spectral path also tries half and
        twice the segment length its cost model picks, and each float32
        plan the other inverse-FFT pass plan (radix 8 / 16) where it can
        take it."""
        gfs, S, hop = g["key"]
        key = (f"{gpu}|{gfs:g}|{S}|{hop}|{length_bucket(g['max_len'])}|{self.accuracy}"
               f"|{self.mode}")
        if self.cache is not None:
            hit = self.cache.get(key)
            if hit:
                return (hit["path"], hit["precision"], int(hit.get("seg_len", 0)),
                        int(hit.get("radix", 0)))
        best = None
        cands = WORKLIST_CANDIDATES if self.mode == "worklist" else CANDIDATES[self.accuracy]
        for path, prec in cands:
            segs = [0]
            while segs:
                seg = segs.pop(0)
                try:
                    plan = self._plan(g, path, prec, seg)
                except cwth.CwthError:
                    continue
                info = plan.info()
                if seg == 0 and path in ("spectral", "auto") and prec == "fp32" and \
                        info["seg_len"] > 0:
                    segs = [m for m in (info["seg_len"] // 2, info["seg_len"] * 2)
                            if 512 <= m <= 32768]
                radices = [0]
                if prec == "fp32" and info["inverse_radix"]:
                    radices.append(8 if info["inverse_radix"] == 16 else 16)
                for radix in radices:
                    if radix:
                        try:
                            plan.set_inverse_radix(radix)
                        except cwth.CwthError:
                            continue
                    ms = self._time(plan, g)
                    if best is None or ms < best[4]:
                        best = (path, prec, seg, radix, ms)
                plan.close()
        if best is None:
            raise cwth.CwthError(4, f"no evaluation serves group {g['key']}")
        if self.cache is not None:
            self.cache.put(key, {"path": best[0], "precision": best[1], "seg_len": best[2],
                                 "radix": best[3], "ms": best[4]})
        return best[0], best[1], best[2], best[3]

    def _time(self, plan, g, reps: int = 3) -> float:
        torch = self.torch
        out = torch.empty((len(g["idx"]), len(g["scales"]), plan.frames_max), device=self.device)
        plan.execute(g["x"], lengths=g["len_d"], out=out)
        plan.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.execute(g["x"], lengths=g["len_d"], out=out)
        e1.record()
        plan.sync()
        return e0.elapsed_time(e1) / reps

    # ------------------------------------------------------------ running
    def run(self):
        """All groups, eagerly, on the current stream: one kernel launch in
        the work-list mode (plus an execute per group the work list cannot
        take), one execute per group in the graph mode."""
        if self.batch is not None:
            self.batch.execute()
        for g in self.solo:
            g["plan"].execute(g["x"], lengths=g["len_d"], out=g["out"])

    def capture(self):
        """Warm up (grows every plan's workspace), then capture all groups into
        one CUDA graph."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self.run()
        self.stream.synchronize()
        for g in self.groups:
            g["plan"].sync()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.run()
        return self.graph

    def replay(self):
        """One launch of the captured graph, on the runner's stream."""
        if self.graph is None:
            self.capture()
        with self.torch.cuda.stream(self.stream):
            self.graph.replay()

    def result(self, i: int) -> np.ndarray:
        """|W| of clip i, [S_i, ceil(len_i / hop_i)] float32 (host copy)."""
        self.stream.synchronize()
        gi, r = self.where[i]
        g = self.groups[gi]
        F = -(-int(g["lens"][r]) // g["key"][2])
        return g["out"][r, :, :F].cpu().numpy()

    def audio_seconds(self) -> float:
        return float(sum(int(g["lens"].sum()) / g["key"][0] for g in self.groups))

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for g in self.groups:
            g["plan"].close()


def uneven_workload(n_clips: int = 1000, seed: int = 2000, min_s: float = 1.0,
                    max_s: float = 30.0, p48k: float = 0.1, scale_counts=(64, 128),
                    hops=(128, 256, 512)):
    """Uneven-length machine-sound clips: lengths uniform in [min_s, max_s]
    seconds, 48 kHz with probability p48k (else 16 kHz), scale count and hop
    drawn uniformly from the given sets.  Clip i uses seed `seed + i`."""
    rng = np.random.default_rng(seed)
    clips, fs, ns, hs = [], [], [], []
    for i in range(n_clips):
        f = 48000.0 if rng.random() < p48k else 16000.0
        n = int(round(rng.uniform(min_s, max_s) * f))
        clips.append(signals.machine_clip(seed + i, n, f))
        fs.append(f)
        ns.append(int(rng.choice(scale_counts)))
        hs.append(int(rng.choice(hops)))
    return clips, fs, ns, hs


def main(argv=None):
    """Time the uneven-length workload as one CUDA-graph launch:
    python -m paper_2408_14302_gb300.batching [--clips 1000] [--reps 5]"""
    import argparse
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--clips", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--accuracy", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--cache", default=None)
    ap.add_argument("--mode", default=None, choices=["worklist", "graph"])
    a = ap.parse_args(argv)
    import torch
    t0 = time.time()
    clips, fs, ns, hs = uneven_workload(a.clips)
    t1 = time.time()
    runner = BatchRunner(clips, fs, ns, hs, accuracy=a.accuracy, cache=TuneCache(a.cache),
                         mode=a.mode)
    t2 = time.time()
    runner.capture()
    runner.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(runner.stream):
        e0.record()
        for _ in range(a.reps):
            runner.graph.replay()
        e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    audio = runner.audio_seconds()
    print(json.dumps({"workload": f"uneven_{a.clips}clips_1-30s_16k48k_S64-128_H128-512",
                      "mode": runner.mode, "groups": len(runner.groups),
                      "work_items": runner.batch.items if runner.batch is not None else None,
                      "audio_seconds": audio,
                      "ms_per_graph_launch": ms, "audio_sec_per_s": audio / (ms * 1e-3),
                      "choices": {str(g["key"]): g["choice"] for g in runner.groups},
                      "generate_s": t1 - t0, "plan_tune_s": t2 - t1}))
    runner.close()


if __name__ == "__main__":
    main()
