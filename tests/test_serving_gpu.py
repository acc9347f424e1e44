"""The continuous-batching server on the GPU: every request's scalogram is
the same in the mix as alone (within 1e-5 of max|W|) and matches the float64
oracle.  The float32 form is held to 1e-5 of max|W|; split bf16 to 1e-5 of
max(max|W|, M), M the largest tap-product mass sum_t |x[kH+t] g[t]| over the
clip's frames, because its error is bounded by about 2^-17 of that mass (the
two bounds coincide unless a short clip makes the sum cancel heavily)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def tap_mass(x, scales, hop, bandwidth=1.5):
    """max over scales and frames of sum_t |x[kH + t]| |g_s[t]| (float64)."""
    x = np.abs(np.asarray(x, np.float64))
    best = 0.0
    for a in scales:
        h = int(np.ceil(a * np.sqrt(bandwidth * np.log(1e16))))
        t = np.arange(-h, h + 1)
        g = np.exp(-(t / a) ** 2 / bandwidth) / np.sqrt(a * np.pi * bandwidth)
        m = np.convolve(x, g, mode="full")[h: h + len(x)]   # centred at each sample
        best = max(best, float(m[::hop].max()))
    return best


@pytest.mark.parametrize("precision,path", [("bf16x2", "auto"), ("fp32", "spectral")])
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
        norm = np.max(ref)
        if precision == "bf16x2":
            norm = max(norm, tap_mass(q.x, sc, q.hop))
        assert np.max(np.abs(got - ref)) <= 1e-5 * norm, q.rid
