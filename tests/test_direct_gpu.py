"""GPU parity of the direct (time-domain GEMM) path against the float64 oracle.

Tolerances, max |err| / max|W| per clip: bf16 operands 2e-2, split hi+lo bf16
1e-5 (where the tap products do not cancel: its bound is about 2^-17 of
the sum of |x g|), split hi+mid+lo bf16 1e-5 on every input, float32 (SIMT)
1e-5.  Workload: the tones generator, 1 s at 16 kHz,
128 scales 100-8000 Hz, hops 64/128/256/512 (the precision study), plus
ragged batches and small hops that exercise overlapping frame views.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16": 2e-2, "bf16x2": 1e-5, "bf16x3": 1e-5, "fp32": 1e-5}


@pytest.fixture(scope="module")
def cw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_14302_gb300 import cwth
    return cwth


@pytest.fixture(scope="module")
def sig():
    from paper_2408_14302_gb300 import signals
    return signals


def oracle_mag(x, scales, hop):
    import oracle
    return oracle.cwth_magnitude(np.asarray(x, np.float32).astype(np.float64), scales, hop)


def run(cw, xs, scales, hop, precision, path="direct", lengths=None, fill=np.nan):
    xs = np.ascontiguousarray(np.atleast_2d(np.asarray(xs, np.float32)))
    with cw.Plan(scales, hop=hop, max_len=xs.shape[1], precision=precision, path=path) as plan:
        out = torch.full((xs.shape[0], len(scales), plan.frames_max), float(fill), device="cuda")
        ld = torch.from_numpy(np.asarray(lengths, np.int64)).cuda() if lengths is not None else None
        plan.execute(torch.from_numpy(xs).cuda(), lengths=ld, out=out)
        plan.sync()
        return out.cpu().numpy().astype(np.float64), plan.info(), plan.scale_paths()


@pytest.mark.parametrize("precision", ["bf16", "bf16x2", "bf16x3", "fp32"])
@pytest.mark.parametrize("hop", [64, 128, 256, 512])
def test_precision_study_128_scales(cw, sig, hop, precision):
    x = sig.tones_clip(seed=0, n=16000).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 128, 16000.0)
    got, info, paths = run(cw, x, sc, hop, precision)
    assert info["num_direct"] == 128 and (paths == 2).all()
    ref = oracle_mag(x, sc, hop)
    err = np.max(np.abs(got[0] - ref)) / ref.max()
    assert err <= TOL[precision], (hop, precision, err)


@pytest.mark.parametrize("precision", ["bf16", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("hop", [8, 16, 40])
def test_small_hops_overlapping_frames(cw, sig, hop, precision):
    x = sig.machine_clip(seed=3, n=6001)
    sc = sig.scales_for_band(200, 8000, 24, 16000.0)
    got, _, _ = run(cw, x, sc, hop, precision)
    ref = oracle_mag(x, sc, hop)
    assert np.max(np.abs(got[0] - ref)) / ref.max() <= TOL[precision]


@pytest.mark.parametrize("precision", ["bf16x2", "bf16x3", "fp32"])
def test_ragged_batch_and_untouched_tail(cw, sig, precision):
    hop, n = 64, 12000
    lengths = [12000, 11999, 1, 0, 500, 64, 65, 7000, 3333]
    xs = np.stack([sig.machine_clip(200 + i, n) for i in range(len(lengths))])
    sc = sig.scales_for_band(100, 8000, 40, 16000.0)
    got, _, _ = run(cw, xs, sc, hop, precision, lengths=lengths, fill=-3.0)
    for i, L in enumerate(lengths):
        F = -(-L // hop)
        assert np.all(got[i, :, F:] == -3.0)
        if L == 0:
            continue
        ref = oracle_mag(xs[i, :L], sc, hop)
        assert np.max(np.abs(got[i, :, :F] - ref)) / ref.max() <= TOL[precision], i


def test_auto_bf16_mixes_paths(cw, sig):
    # Scales with more than 4096 taps go to the spectral path.
    x = sig.machine_clip(seed=4, n=40000)
    sc = np.array([2.0, 5.0, 30.0, 200.0, 500.0, 1200.0])
    got, info, paths = run(cw, x, sc, 64, "bf16x2", path="auto")
    assert info["num_direct"] >= 3 and info["num_spectral"] >= 1
    assert paths[0] == 2 and paths[-1] == 1
    ref = oracle_mag(x, sc, 64)
    assert np.max(np.abs(got[0] - ref)) / ref.max() <= 1e-5


def test_direct_large_batch_sampled(cw, sig):
    """512 clips (the precision study's throughput batch), rows sampled."""
    hop = 64
    xs = np.stack([sig.tones_clip(seed=s, n=16000) for s in range(512)]).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 128, 16000.0)
    got, _, _ = run(cw, xs, sc, hop, "bf16x2")
    assert np.isfinite(got).all()
    for i in (0, 255, 511):
        ref = oracle_mag(xs[i], sc, hop)
        assert np.max(np.abs(got[i] - ref)) / ref.max() <= 1e-5


def tap_mass(x, scales, hop):
    """Largest sum of |x[kH + t] g_s[t]| over the frames and scales (float64,
    the same taps as the oracle): the quantity a split's per-product error
    is relative to."""
    x = np.abs(np.asarray(x, np.float64))
    best = 0.0
    for a in scales:
        h = int(np.ceil(a * np.sqrt(1.5 * np.log(1e16))))
        t = np.arange(-h, h + 1) / a
        g = np.exp(-t * t / 1.5) / np.sqrt(a * np.pi * 1.5)
        m = np.convolve(x, g, mode="full")[h:h + len(x)]
        best = max(best, float(m[::hop].max()))
    return best


def test_cancelling_short_clip_split_precisions(cw):
    """A short white-noise clip with long wavelets: each scalogram value is a
    sum of up to ~3600 tap products of random sign, so the tap-product mass
    is several times max|W|.

    * The automatic three-part split plan (tensor cores for supports up to
      1024 padded taps, float32 spectral beyond) holds 1e-5 of max|W|.
    * Forced onto the tensor cores, the three-part split holds 1e-5 on
      every row up to 1024 taps; longer rows carry the float32
      accumulation's bias (about 1e-5 relative at 2300 taps), bounded
      here by 3e-5.
    * The two-part split holds its own bound, 2^-16 of the tap-product
      mass."""
    rng = np.random.default_rng(12)
    x = rng.standard_normal(8000).astype(np.float32)
    sc = np.geomspace(2.0, 320.0, 24)
    ref = oracle_mag(x, sc, 64)
    mass = tap_mass(x, sc, 64)
    assert mass > 5 * ref.max()   # 2^-17 of the mass is then above 1e-5 of max|W|
    got, info, paths = run(cw, x, sc, 64, "bf16x3", path="auto")
    assert info["num_direct"] > 0 and info["num_spectral"] > 0, info
    assert np.max(np.abs(got[0] - ref)) / ref.max() <= 1e-5
    got3, info3, _ = run(cw, x, sc, 64, "bf16x3")
    short = np.array([2 * int(np.ceil(a * np.sqrt(1.5 * np.log(1e9)))) + 1 <= 1024 for a in sc])
    err3 = np.max(np.abs(got3[0] - ref), axis=1) / ref.max()
    assert np.all(err3[short] <= 1e-5) and np.all(err3 <= 3e-5), err3
    got2, _, _ = run(cw, x, sc, 64, "bf16x2")
    assert np.max(np.abs(got2[0] - ref)) <= 2.0 ** -16 * mass


def test_bf16x3_auto_and_large_batch(cw, sig):
    """The three-part split through the automatic path (scales beyond 4096
    taps go spectral) and on the 512-clip throughput batch, rows sampled."""
    x = sig.machine_clip(seed=4, n=40000)
    sc = np.array([2.0, 5.0, 30.0, 200.0, 500.0, 1200.0])
    got, info, paths = run(cw, x, sc, 64, "bf16x3", path="auto")
    assert info["num_direct"] >= 3 and info["num_spectral"] >= 1
    ref = oracle_mag(x, sc, 64)
    assert np.max(np.abs(got[0] - ref)) / ref.max() <= 1e-5
    xs = np.stack([sig.tones_clip(seed=s, n=16000) for s in range(512)]).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 128, 16000.0)
    got, _, _ = run(cw, xs, sc, 64, "bf16x3")
    for i in (0, 511):
        ref = oracle_mag(xs[i], sc, 64)
        assert np.max(np.abs(got[i] - ref)) / ref.max() <= 1e-5


def test_direct_unsupported_cases(cw):
    with pytest.raises(cw.CwthError):
        cw.Plan([2.0], hop=12, max_len=1000, precision="bf16", path="direct")   # hop % 8
    with pytest.raises(cw.CwthError):
        cw.Plan([900.0], hop=64, max_len=1000, precision="bf16", path="direct")  # > 4096 taps


def test_reserve_moves_workspace_growth_out_of_execute(cw, sig):
    """cwth_plan_reserve sizes the staged bf16 signal (and the host
    pipeline's staging) up front: after it, executes of up to that many
    clips leave the device's free memory unchanged, and give the same bytes
    as a plan that grew its workspace inside execute."""
    n, hop, B = 32000, 64, 48
    sc = sig.scales_for_band(100, 8000, 48, 16000.0)
    xh = np.ascontiguousarray(sig.machine_batch(B, n))
    xs = torch.from_numpy(xh).cuda()

    def one(reserve):
        with cw.Plan(sc, hop=hop, max_len=n, precision="bf16x2", path="direct") as plan:
            out = torch.empty((B, len(sc), plan.frames_max), device="cuda")
            # One clip first, so every kernel is loaded before memory is read.
            plan.execute(xs[:1], out=out[:1])
            plan.sync()
            if reserve:
                plan.reserve(B, ld_x=n, host=True)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            for b in (16, B, 32):
                plan.execute(xs[:b], out=out[:b])
            plan.sync()
            free1 = torch.cuda.mem_get_info()[0]
            if reserve:
                h_out = np.empty((B, len(sc), plan.frames_max), np.float32)
                plan.execute_host(xh, h_out)
                assert torch.cuda.mem_get_info()[0] == free1
                assert np.array_equal(h_out, out.cpu().numpy())
            return out.cpu().numpy(), free0 - free1

    got, grew = one(True)
    ref, grew_plain = one(False)
    assert grew == 0, grew
    # Control: without the reservation the same calls allocate (48 clips of
    # 32000 samples staged as two bf16 parts are about 6 MB).
    assert grew_plain > 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_staging_alignment_does_not_change_results(cw, sig, precision):
    """The bf16 staging reads 16-byte-aligned interior runs as float4 and
    everything else element by element; a batch whose rows are offset by
    one float (no float4 reads) and one with an odd row stride give the
    aligned batch's scalograms byte for byte."""
    hop, n = 64, 9001
    lengths = [9001, 8999, 4097, 1]
    xs = np.stack([sig.machine_clip(300 + i, n) for i in range(len(lengths))]).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 24, 16000.0)
    ld = torch.tensor(lengths, dtype=torch.int64, device="cuda")
    with cw.Plan(sc, hop=hop, max_len=n, precision=precision, path="direct") as plan:
        outs = []
        wide = torch.zeros((len(lengths), n + 3), device="cuda")
        wide[:, 1:n + 1] = torch.from_numpy(xs).cuda()
        for x in (torch.from_numpy(xs).cuda(),   # ld_x = 9001 (odd)
                  wide[:, 1:n + 1]):             # base one float past 16-byte alignment
            out = torch.full((len(lengths), len(sc), plan.frames_max), -1.0, device="cuda")
            plan.execute(x, lengths=ld, out=out)
            outs.append(out)
        plan.sync()
        # the aligned reference: rows of 9004 floats, base aligned (the
        # staged signal's front padding is a multiple of 8 samples)
        al = torch.zeros((len(lengths), n + 3), device="cuda")
        al[:, :n] = torch.from_numpy(xs).cuda()
        ref = torch.full_like(outs[0], -1.0)
        plan.execute(al[:, :n], lengths=ld, out=ref)
        plan.sync()
    for out in outs:
        assert torch.equal(out, ref)
    F = -(-lengths[0] // hop)
    assert np.max(np.abs(ref[0, :, :F].cpu().numpy() - oracle_mag(xs[0], sc, hop))) / \
        float(ref[0].max()) <= TOL[precision]


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_bound_staging_buffer_gives_identical_results(cw, sig, precision):
    """A plan staging its bf16 signal in caller-bound buffers (one per
    stream, as the server's slots do) gives the plan-owned staging's
    scalograms byte for byte, across two buffers used in turn, with two GEMM
    groups (200 scales); a buffer too small for the batch is refused before
    anything is enqueued."""
    hop, n = 64, 12000
    lengths = [12000, 7001, 1]
    xs = np.stack([sig.machine_clip(400 + i, n) for i in range(len(lengths))]).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 200, 16000.0)
    x = torch.from_numpy(xs).cuda()
    ld = torch.tensor(lengths, dtype=torch.int64, device="cuda")
    with cw.Plan(sc, hop=hop, max_len=n, precision=precision, path="direct") as plan:
        ref = torch.full((len(lengths), len(sc), plan.frames_max), -4.0, device="cuda")
        plan.execute(x, lengths=ld, out=ref)
        need = plan.stage_bytes(len(lengths))
        assert need > 0
        bufs = [torch.empty(need + 512 * k, dtype=torch.uint8, device="cuda") for k in range(2)]
        for buf in bufs + bufs:
            plan.bind_stage(buf)
            out = torch.full_like(ref, -4.0)
            plan.execute(x, lengths=ld, out=out)
            plan.sync()
            assert torch.equal(out, ref)
        small = torch.empty(need - 4096, dtype=torch.uint8, device="cuda")
        plan.bind_stage(small)
        out = torch.full_like(ref, -4.0)
        with pytest.raises(cw.CwthError):
            plan.execute(x, lengths=ld, out=out)
        plan.sync()
        assert bool((out == -4.0).all())
        plan.bind_stage(None)
        plan.execute(x, lengths=ld, out=out)
        plan.sync()
        assert torch.equal(out, ref)
