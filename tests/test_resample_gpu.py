"""Resample-first reading of the hop (cwth_plan_resampled) against the
float64 oracle: y[m] = x[m H], then the CWT at every sample of y with scales
a / H.  Tolerance: max |err| <= 1e-5 * max|W| per clip (float32 path)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def cw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth
    return cwth


def _check_clip(oracle, got, x, sc, hop, L):
    ref = np.abs(oracle.cwth_resampled(np.asarray(x[:L], np.float64), sc, hop))
    F = ref.shape[1]
    err = float(np.max(np.abs(got[:, :F] - ref))) / max(float(ref.max()), 1e-30)
    assert err <= TOL, (hop, L, err)


@pytest.mark.parametrize("hop,f_lo,f_hi", [(2, 100, 4000), (8, 100, 1000), (64, 50, 125)])
def test_resampled_plan_matches_oracle(cw, hop, f_lo, f_hi):
    import oracle
    from paper_2408_14302_gb300 import signals
    n, B = 24000, 3
    xs = np.stack([signals.machine_clip(60 + i, n) for i in range(B)]).astype(np.float32)
    sc = signals.scales_for_band(f_lo, f_hi, 12, 16000.0)
    lens = np.array([n, 7777, 1], np.int64)
    with cw.Plan(sc, hop=hop, max_len=n, resample_first=True) as plan:
        info = plan.info()
        assert info["resample"] == hop and info["hop"] == 1
        assert plan.frames_max == -(-n // hop)
        x = torch.from_numpy(xs).cuda()
        out = plan.execute(x).cpu().numpy()
        for i in range(B):
            _check_clip(oracle, out[i], xs[i], sc, hop, n)
        # per-clip lengths: frames past ceil(len / H) stay untouched
        o2 = torch.full((B, len(sc), plan.frames_max), -3.0, device="cuda")
        plan.execute(x, lengths=torch.from_numpy(lens).cuda(), out=o2)
        o2 = o2.cpu().numpy()
        for i, L in enumerate(lens):
            F = -(-int(L) // hop)
            assert np.all(o2[i, :, F:] == -3.0)
            _check_clip(oracle, o2[i], xs[i], sc, hop, int(L))
        # the host entry point gives the same bytes for any chunk count
        for chunks in (1, 2, 3):
            plan.set_host_chunks(chunks)
            h = np.full((B, len(sc), plan.frames_max), -3.0, np.float32)
            plan.execute_host(xs, h, lengths=lens)
            assert np.array_equal(h, o2), chunks


def test_resampled_split_bf16_plan(cw):
    # bf16 operands need a hop that is a multiple of 8, so the hop-1
    # transform of the re-sampled signal takes the float32 spectral path.
    import oracle
    from paper_2408_14302_gb300 import signals
    n = 16000
    x = signals.tones_clip(seed=5, n=n).astype(np.float32)
    sc = signals.scales_for_band(100, 2000, 10, 16000.0)
    with cw.Plan(sc, hop=4, max_len=n, precision="bf16x2", resample_first=True) as plan:
        assert plan.info()["num_spectral"] == len(sc)
        got = plan.execute(torch.from_numpy(x).cuda()).cpu().numpy()[0]
    _check_clip(oracle, got, x, sc, 4, n)
