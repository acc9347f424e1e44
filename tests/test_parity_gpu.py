"""GPU parity: libcwth.so (through the C ABI) against the float64 oracle.

Tolerance (float32 spectral path): max |err| <= 1e-5 * max|W| per clip, the
normaliser taken over all scales and frames of that clip.  The oracle sees
the same float32 samples the GPU sees, promoted to float64.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


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


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(ref))


def run_gpu(cw, x, scales, hop, lengths=None, path="auto", precision="fp32", max_len=None,
            fill=np.nan):
    x = np.ascontiguousarray(np.atleast_2d(np.asarray(x, np.float32)))
    max_len = x.shape[1] if max_len is None else max_len
    with cw.Plan(scales, hop=hop, max_len=max_len, path=path, precision=precision) as plan:
        xd = torch.from_numpy(x).cuda()
        out = torch.full((x.shape[0], len(scales), plan.frames_max), float(fill),
                         dtype=torch.float32, device="cuda")
        ld = torch.from_numpy(np.asarray(lengths, np.int64)).cuda() if lengths is not None else None
        plan.execute(xd, lengths=ld, out=out)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64), plan.info()


def oracle_mag(x, scales, hop):
    import oracle
    return oracle.cwth_magnitude(np.asarray(x, np.float32).astype(np.float64), scales, hop)


@pytest.mark.parametrize("hop", [64, 1])
def test_tones_1s_32_scales(cw, sig, hop):
    x = sig.tones_clip(seed=0, n=16000).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 32, 16000.0)
    got, info = run_gpu(cw, x, sc, hop)
    ref = oracle_mag(x, sc, hop)
    assert got.shape == (1, 32, ref.shape[1])
    assert rel_err(got[0], ref) <= TOL_FP32, info


@pytest.mark.parametrize("hop", [2, 8, 32, 128, 256, 512, 1024])
def test_hops_ragged_tail(cw, sig, hop):
    # 9000 samples: not a multiple of any of these hops (ragged last frame),
    # several segments per clip.
    x = sig.machine_clip(seed=5, n=9001, dtype=np.float32)
    sc = sig.scales_for_band(50, 8000, 12, 16000.0)
    got, info = run_gpu(cw, x, sc, hop)
    ref = oracle_mag(x, sc, hop)
    assert info["num_segments"] >= 1
    assert rel_err(got[0], ref) <= TOL_FP32, info


def test_machine_10s_64_scales_hop256_full_clips(cw, sig):
    n, hop = 160000, 256
    xs = np.stack([sig.machine_clip(1000 + i, n) for i in range(3)])
    sc = sig.scales_for_band(50, 8000, 64, 16000.0)
    got, info = run_gpu(cw, xs, sc, hop)
    assert info["num_segments"] > 1
    for i in range(3):
        ref = oracle_mag(xs[i], sc, hop)
        assert rel_err(got[i], ref) <= TOL_FP32


def test_machine_batch64_sampled_rows(cw, sig):
    """Full 64-clip batch in the benchmark's launch configuration; rows of a
    few clips and scales are checked against the oracle one by one."""
    n, hop, B = 160000, 256, 64
    xs = sig.machine_batch(B, n)
    sc = sig.scales_for_band(50, 8000, 64, 16000.0)
    got, _ = run_gpu(cw, xs, sc, hop)
    assert np.isfinite(got).all()
    rng = np.random.default_rng(0)
    for i in (0, 31, 63):
        rows = np.sort(rng.choice(64, 6, replace=False))
        ref = oracle_mag(xs[i], sc[rows], hop)
        # normaliser: max|W| of the clip over all scales (largest scales dominate)
        ref_full_max = max(float(ref.max()), float(oracle_mag(xs[i], sc[-4:], hop).max()))
        err = float(np.max(np.abs(got[i, rows] - ref))) / ref_full_max
        assert err <= TOL_FP32


def test_forced_segment_lengths_agree(cw, sig):
    """cwth_plan_segment: every valid segment length gives the oracle's
    scalogram (each one evaluates the linear correlation of Eq. 1 at its
    frames), and an unusable one is refused."""
    n, hop = 20000, 64
    x = sig.machine_clip(31, n)
    sc = sig.scales_for_band(50, 8000, 24, 16000.0)
    ref = oracle_mag(x, sc, hop)
    xd = torch.from_numpy(np.asarray(x, np.float32)[None]).cuda()
    for seg in (4096, 8192, 16384):
        with cw.Plan(sc, hop=hop, max_len=n, path="spectral", seg_len=seg) as plan:
            assert plan.info()["seg_len"] == seg
            got = plan.execute(xd).cpu().numpy()[0].astype(np.float64)
        assert rel_err(got, ref) <= TOL_FP32, seg
    with pytest.raises(cw.CwthError):
        # 512 samples hold no valid frame next to the 50 Hz wavelet's support
        cw.Plan(sc, hop=hop, max_len=n, path="spectral", seg_len=512)


def test_pruned_inverse_ffts_several_scales_per_pass(cw, sig):
    """Hop 1 on a short clip with narrow Morlet bands (200-2000 Hz): the plan
    takes the pruned kernel (leading inverse-FFT passes skipped) with
    several scales per pass, so each chunk's pruning bound comes from the
    suffix maximum of its band widths.  Scales are given in descending order
    to check that the plan's internal ascending order keeps every output
    row in the caller's order."""
    n, hop = 3000, 1
    x = sig.tones_clip(7, n)
    sc = sig.scales_for_band(200, 2000, 16, 16000.0)[::-1].copy()
    got, info = run_gpu(cw, x, sc, hop)
    assert info["spectral_pruned"] == 1 and info["spectral_pass_scales"] > 1, info
    ref = oracle_mag(x, sc, hop)
    assert rel_err(got[0], ref) <= TOL_FP32


@pytest.mark.parametrize("hop", [1, 4, 8, 512, 1024])
def test_machine_10s_sampled_scales(cw, sig, hop):
    """Full 10 s clips in the benchmark's 64-scale plan at hop 1 (the
    metric's comparison point), hops 4 and 8 (inverse FFTs of 4096 and 2048
    points, one or two scales per pass) and hops 512 and 1024 (periods of 32
    and 16 residues: one fold warp covers one or two scales); the widest, a
    middle and the narrowest scale rows are checked against the oracle,
    normalised by their own maximum (stricter than the maximum over all
    scales)."""
    n = 160000
    xs = sig.machine_batch(2, n)
    sc = sig.scales_for_band(50, 8000, 64, 16000.0)
    got, info = run_gpu(cw, xs, sc, hop)
    assert info["num_segments"] > 1 and got.shape[2] == -(-n // hop)
    rows = np.array([0, 31, 63])
    for i in range(2):
        ref = oracle_mag(xs[i], sc[rows], hop)
        err = float(np.max(np.abs(got[i, rows] - ref))) / float(ref.max())
        assert err <= TOL_FP32, (i, err)


def test_ragged_lengths_and_untouched_tail(cw, sig):
    hop, n = 64, 20000
    lengths = [20000, 19999, 1, 0, 777, 64, 65, 12345]
    xs = np.stack([sig.machine_clip(50 + i, n) for i in range(len(lengths))])
    sc = sig.scales_for_band(50, 8000, 16, 16000.0)
    got, _ = run_gpu(cw, xs, sc, hop, lengths=lengths, fill=-7.0)
    for i, L in enumerate(lengths):
        F = -(-L // hop)
        assert np.all(got[i, :, F:] == -7.0), f"clip {i}: frames beyond ceil(len/H) written"
        if L == 0:
            continue
        ref = oracle_mag(xs[i, :L], sc, hop)
        assert rel_err(got[i, :, :F], ref) <= TOL_FP32, f"clip {i} (len {L})"


def test_single_scale_small_and_large(cw, sig):
    x = sig.tones_clip(seed=2, n=3000).astype(np.float32)
    for sc in ([0.7], [2.0], [400.0], [1.1, 600.0]):
        sc = np.asarray(sc)
        got, _ = run_gpu(cw, x, sc, 16)
        ref = oracle_mag(x, sc, 16)
        assert rel_err(got[0], ref) <= TOL_FP32, sc


def test_other_morlet_parameters(cw, sig):
    import oracle
    x = sig.tones_clip(seed=3, n=5000).astype(np.float32)
    sc = sig.scales_for_band(100, 8000, 10, 16000.0)
    for B, C in ((1.0, 1.5), (2.0, 0.8)):
        with cw.Plan(sc, hop=32, max_len=5000, bandwidth=B, center=C) as plan:
            out = plan.execute(torch.from_numpy(x).cuda().unsqueeze(0))
            got = out[0].cpu().numpy().astype(np.float64)
        ref = np.abs(oracle.cwth(x.astype(np.float64), sc, 32, bandwidth=B, center=C))
        assert rel_err(got, ref) <= TOL_FP32


def test_host_entry_point_matches_device(cw, sig):
    n, hop = 30000, 128
    xs = np.stack([sig.machine_clip(70 + i, n) for i in range(4)]).astype(np.float32)
    sc = sig.scales_for_band(50, 8000, 20, 16000.0)
    with cw.Plan(sc, hop=hop, max_len=n) as plan:
        dev = plan.execute(torch.from_numpy(xs).cuda()).cpu().numpy()
        hx = torch.from_numpy(xs).pin_memory()
        hout = torch.empty((4, 20, plan.frames_max), dtype=torch.float32).pin_memory()
        plan.execute_host(hx, hout)
        assert np.array_equal(hout.numpy(), dev)
        lens = np.array([n, 100, 0, 29999], np.int64)
        hout2 = np.full((4, 20, plan.frames_max), -1.0, np.float32)
        plan.execute_host(xs, hout2, lengths=lens)
        for i, L in enumerate(lens):
            F = -(-int(L) // hop)
            assert np.all(hout2[i, :, F:] == -1.0)
        assert np.array_equal(hout2[0], dev[0])


def test_host_pipeline_chunks_do_not_change_results(cw, sig):
    # cwth_execute_host overlaps the upload, transform and download of clip
    # chunks; every chunk count must give the device path's exact bytes,
    # with and without lengths, on the spectral and the direct path.
    n, hop, B = 20000, 64, 7
    xs = np.stack([sig.machine_clip(90 + i, n) for i in range(B)]).astype(np.float32)
    lens = np.array([n, 1, 0, 12345, n - 1, 64, 9000], np.int64)
    sc = sig.scales_for_band(60, 7000, 24, 16000.0)
    hx = torch.from_numpy(xs).pin_memory()
    for precision in ("fp32", "bf16x2"):
        with cw.Plan(sc, hop=hop, max_len=n, precision=precision) as plan:
            dev = plan.execute(torch.from_numpy(xs).cuda()).cpu().numpy()
            dl = torch.from_numpy(lens).cuda()
            devl = torch.full((B, len(sc), plan.frames_max), -1.0, device="cuda")
            plan.execute(torch.from_numpy(xs).cuda(), lengths=dl, out=devl)
            devl = devl.cpu().numpy()
            for chunks in (0, 1, 2, 3, 7, 50):
                plan.set_host_chunks(chunks)
                hout = torch.empty((B, len(sc), plan.frames_max), dtype=torch.float32).pin_memory()
                plan.execute_host(hx, hout)
                assert np.array_equal(hout.numpy(), dev), (precision, chunks)
                hout2 = np.full((B, len(sc), plan.frames_max), -1.0, np.float32)
                plan.execute_host(xs, hout2, lengths=lens)
                assert np.array_equal(hout2, devl), (precision, chunks)


def test_non_default_stream_and_two_plans(cw, sig):
    n = 12000
    x = torch.from_numpy(sig.machine_clip(9, n)).cuda().unsqueeze(0)
    sc1 = sig.scales_for_band(50, 8000, 8, 16000.0)
    sc2 = sig.scales_for_band(200, 4000, 5, 16000.0)
    with cw.Plan(sc1, hop=64, max_len=n) as p1, cw.Plan(sc2, hop=32, max_len=n) as p2:
        ref1 = p1.execute(x).clone()
        ref2 = p2.execute(x).clone()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            o1 = p1.execute(x)
            o2 = p2.execute(x)
        s.synchronize()
        assert torch.equal(o1, ref1) and torch.equal(o2, ref2)


def test_deterministic(cw, sig):
    x = torch.from_numpy(sig.machine_batch(4, 40000)).cuda()
    sc = sig.scales_for_band(50, 8000, 32, 16000.0)
    with cw.Plan(sc, hop=256, max_len=40000) as plan:
        a = plan.execute(x).clone()
        b = plan.execute(x)
        assert torch.equal(a, b)


def test_cost_model_split_fused_scales(cw, sig):
    """Automatic float32 plans: the cost model sends the short-support
    scales (wide Morlet bands, whose hop fold costs about H/a bins per
    frame) to the spectral kernel's time-domain phase.  The fused scales are
    the smallest ones; the result matches the oracle, including ragged
    lengths, and so does the all-spectral plan of the same scales."""
    n, hop = 40000, 256
    lengths = [40000, 39999, 257, 0, 30001]
    xs = np.stack([sig.machine_clip(400 + i, n) for i in range(len(lengths))])
    sc = sig.scales_for_band(50, 8000, 64, 16000.0)
    got, info = run_gpu(cw, xs, sc, hop, lengths=lengths, fill=-3.0)
    assert info["num_fused"] > 0 and info["num_spectral"] > 0, info
    assert info["num_direct"] == info["num_fused"]
    with cw.Plan(sc, hop=hop, max_len=n) as p:
        paths = p.scale_paths()
    fused = paths == 2
    assert fused.sum() == info["num_fused"] and sc[fused].max() < sc[~fused].min()
    spec, info2 = run_gpu(cw, xs, sc, hop, lengths=lengths, path="spectral", fill=-3.0)
    assert info2["num_fused"] == 0 and info2["num_spectral"] == 64
    for i, L in enumerate(lengths):
        F = -(-L // hop)
        assert np.all(got[i, :, F:] == -3.0) and np.all(spec[i, :, F:] == -3.0)
        if L == 0:
            continue
        ref = oracle_mag(xs[i, :L], sc, hop)
        assert rel_err(got[i, :, :F], ref) <= TOL_FP32, (i, L)
        assert rel_err(spec[i, :, :F], ref) <= TOL_FP32, (i, L)


@pytest.mark.parametrize("hop", [128, 1024])
def test_all_scales_fused(cw, sig, hop):
    """High-frequency scales only, at large hops: every scale is cheaper as
    a direct sum, so the spectral kernel runs its time-domain phase alone
    (no FFT)."""
    n = 30000
    xs = np.stack([sig.machine_clip(77 + i, n) for i in range(2)])
    sc = sig.scales_for_band(2500, 8000, 12, 16000.0)
    got, info = run_gpu(cw, xs, sc, hop)
    assert info["num_fused"] == 12 and info["num_spectral"] == 0, info
    for i in range(2):
        ref = oracle_mag(xs[i], sc, hop)
        assert rel_err(got[i], ref) <= TOL_FP32


def test_1024_thread_shape_hop2_long_segments(cw, sig):
    """Hop 2 with 16384-sample segments: one scale's 8192-point inverse FFT
    does not fit beside the spectrum in the two-CTA shape's shared memory,
    so the plan takes one 1024-thread CTA per SM.  Ragged clips over three
    segments against the oracle."""
    n, hop = 40000, 2
    xs = np.stack([sig.machine_clip(501 + i, n) for i in range(2)])
    lengths = [n, 23457]
    sc = sig.scales_for_band(200, 8000, 24, 16000.0)
    with cw.Plan(sc, hop=hop, max_len=n, path="spectral", seg_len=16384) as plan:
        info = plan.info()
        assert info["spectral_threads"] == 1024 and info["num_segments"] >= 3, info
        out = torch.full((2, len(sc), plan.frames_max), -3.0, device="cuda")
        plan.execute(torch.from_numpy(np.ascontiguousarray(xs, np.float32)).cuda(),
                     lengths=torch.tensor(lengths, dtype=torch.int64, device="cuda"), out=out)
        plan.sync()
        got = out.cpu().numpy().astype(np.float64)
    for i, L in enumerate(lengths):
        F = -(-L // hop)
        ref = oracle_mag(xs[i, :L], sc, hop)
        assert rel_err(got[i, :, :F], ref) <= TOL_FP32, i
        assert np.all(got[i, :, F:] == -3.0)


def test_two_part_plan_hop1(cw, sig):
    """Hop 1 over 50-8000 Hz: the cost model runs the smallest scales as
    further spectral parts with their own short-halo segments.  Rows of both
    parts against the oracle, and the whole scalogram against a one-part
    plan (a forced segment length never splits)."""
    n, hop = 60000, 1
    xs = sig.machine_batch(2, n)
    sc = sig.scales_for_band(50, 8000, 48, 16000.0)
    got, info = run_gpu(cw, xs, sc, hop)
    assert info["spectral_parts"] >= 2 and info["num_spectral"] == 48, info
    with cw.Plan(sc, hop=hop, max_len=n, seg_len=info["seg_len"]) as one:
        assert one.info()["spectral_parts"] == 1
        ref1 = one.execute(torch.from_numpy(xs.astype(np.float32)).cuda()).cpu().numpy()
    rows = np.array([0, 8, 16, 24, 32, 40, 47])
    for i in range(2):
        assert rel_err(got[i], ref1[i]) <= TOL_FP32
        ref = oracle_mag(xs[i], sc[rows], hop)
        err = float(np.max(np.abs(got[i, rows] - ref))) / float(ref.max())
        assert err <= TOL_FP32, (i, err)


@pytest.mark.parametrize("hop", [3, 5, 7, 12, 54, 96, 100, 336, 1600])
def test_non_power_of_two_hops(cw, sig, hop):
    """Hops with an odd factor d (3, 5, 7, 3 * 2^2, 27 * 2, 3 * 2^5, 25 * 2^2,
    21 * 2^4, 25 * 2^6): segments of M = 2 d N2 samples, d column FFTs of
    N2 points plus radix-3/5/7 passes, and the fold at P = M / H.  Forced
    spectral and automatic float32 plans, ragged clips, against the oracle."""
    n = 20000
    xs = np.stack([sig.machine_clip(900 + i, n) for i in range(2)])
    lengths = [n, 13001]
    sc = sig.scales_for_band(50, 8000, 24, 16000.0)
    refs = [oracle_mag(xs[i, :L], sc, hop) for i, L in enumerate(lengths)]
    for path in ("spectral", "auto"):
        got, info = run_gpu(cw, xs, sc, hop, lengths=lengths, path=path, fill=-2.0)
        assert info["num_spectral"] == 24 and info["seg_len"] % hop == 0, info
        d = hop
        while d % 2 == 0:
            d //= 2
        assert (info["seg_len"] // 2) % d == 0 and info["fold_len"] & (info["fold_len"] - 1) == 0
        for i, L in enumerate(lengths):
            F = -(-L // hop)
            assert rel_err(got[i, :, :F], refs[i]) <= TOL_FP32, (path, i)
            assert np.all(got[i, :, F:] == -2.0)


def test_non_power_of_two_hop_forced_segments(cw, sig):
    """Hop 96 (d = 3): every segment length of the form 2 * 3 * 2^k the
    plan accepts gives the oracle's scalogram; one whose odd part is not the
    hop's is refused."""
    n, hop = 30000, 96
    x = sig.machine_clip(41, n)
    sc = sig.scales_for_band(50, 8000, 16, 16000.0)
    ref = oracle_mag(x, sc, hop)
    xd = torch.from_numpy(np.asarray(x, np.float32)[None]).cuda()
    for seg in (6144, 12288):
        with cw.Plan(sc, hop=hop, max_len=n, path="spectral", seg_len=seg) as plan:
            assert plan.info()["seg_len"] == seg
            got = plan.execute(xd).cpu().numpy()[0].astype(np.float64)
        assert rel_err(got, ref) <= TOL_FP32, seg
    with pytest.raises(cw.CwthError) as e:
        cw.Plan(sc, hop=hop, max_len=n, path="spectral", seg_len=5 * 2048)
    assert e.value.status == 4


def test_unsupported_hop_for_spectral(cw):
    """Hop 11 (odd part 11) and hop 2^3 * 45 (odd part 45 > 27) stay with
    the direct path; a forced spectral plan is refused."""
    for hop in (11, 360):
        with pytest.raises(cw.CwthError) as e:
            cw.Plan([2.0, 5.0], hop=hop, max_len=1000, path="spectral")
        assert e.value.status == 4


def test_outputs_stay_inside_their_buffers(cw, sig):
    """Guard bands: every path writes only inside its [batch][S][F_max]
    output (a sentinel before and after it survives, as does the sentinel
    in the frames past each clip) — the automatic float32 plan at hop 256
    (folded and fused scales) and at hop 4 (several spectral parts, pruned
    inverse FFTs), a tensor-core bf16x3 plan, an odd hop, and the host entry
    point."""
    n, G, sent = 30000, 4096, -7.0
    xs = sig.machine_batch(3, n)
    lengths = [n, 17001, 1]
    sc = sig.scales_for_band(50, 8000, 24, 16000.0)
    xd = torch.from_numpy(np.ascontiguousarray(xs, np.float32)).cuda()
    ld = torch.tensor(lengths, dtype=torch.int64, device="cuda")
    for hop, precision in ((256, "fp32"), (4, "fp32"), (64, "bf16x3"), (96, "fp32")):
        with cw.Plan(sc, hop=hop, max_len=n, precision=precision) as plan:
            F = plan.frames_max
            size = 3 * len(sc) * F
            big = torch.full((size + 2 * G,), sent, device="cuda")
            out = big[G:G + size].view(3, len(sc), F)
            plan.execute(xd, lengths=ld, out=out)
            plan.sync()
            h = big.cpu().numpy()
            assert np.all(h[:G] == sent) and np.all(h[G + size:] == sent), (hop, precision)
            o = out.cpu().numpy()
            for i, L in enumerate(lengths):
                assert np.all(o[i, :, -(-L // hop):] == sent), (hop, precision, i)
            assert np.all(np.isfinite(o)) and o[0].max() > 0
    for hop in (128, 96):
        with cw.Plan(sc, hop=hop, max_len=n) as plan:
            F = plan.frames_max
            size = 3 * len(sc) * F
            hbig = np.full(size + 2 * G, sent, np.float32)
            hout = hbig[G:G + size].reshape(3, len(sc), F)
            plan.execute_host(np.ascontiguousarray(xs, np.float32), hout)
            assert np.all(hbig[:G] == sent) and np.all(hbig[G + size:] == sent), hop
            assert np.all(np.isfinite(hout)) and hout.max() > 0
            dev = plan.execute(xd).cpu().numpy()
            assert np.array_equal(dev, hout), hop


def test_inverse_radix_knob(cw, sig):
    """cwth_plan_set_inverse_radix: radix-8 and radix-16 inverse-FFT pass
    plans give the same scalogram within the float32 tolerance (and the
    oracle's); 0 restores the model's choice; a pruned plan refuses 8."""
    n, hop = 30000, 256
    xs = sig.machine_batch(2, n)
    sc = sig.scales_for_band(50, 8000, 24, 16000.0)
    xd = torch.from_numpy(np.ascontiguousarray(xs, np.float32)).cuda()
    with cw.Plan(sc, hop=hop, max_len=n) as p:
        model = p.info()["inverse_radix"]
        assert model in (8, 16)
        outs = {}
        for r in (8, 16):
            p.set_inverse_radix(r)
            assert p.info()["inverse_radix"] == r
            outs[r] = p.execute(xd).cpu().numpy().astype(np.float64)
        p.set_inverse_radix(0)
        assert p.info()["inverse_radix"] == model
    for i in range(2):
        assert rel_err(outs[8][i], outs[16][i]) <= TOL_FP32
        assert rel_err(outs[8][i], oracle_mag(xs[i], sc, hop)) <= TOL_FP32
    with cw.Plan(sc, hop=1, max_len=4000) as p1:
        assert p1.info()["spectral_pruned"] == 1
        with pytest.raises(cw.CwthError) as e:
            p1.set_inverse_radix(8)
        assert e.value.status == 4
        p1.set_inverse_radix(16)


@pytest.mark.parametrize("precision,hop,n", [("fp32", 1, 60000), ("fp32", 8, 60000),
                                             ("bf16x3", 256, 60000)])
def test_dependent_launches_keep_stream_order(cw, sig, precision, hop, n):
    """A plan's later spectral parts (and, with tensor-core scales, its
    spectral part after the tensor-core kernel, which itself follows the
    bf16 staging) start before the kernel before them ends.  Executes queued
    back to back on one stream with no synchronisation, alternating inputs
    and outputs, and stream work that reads each output right after its
    execute, must see every row of every part: each result equals the same
    input transformed alone."""
    xs = [sig.machine_batch(2, n, seed0=s).astype(np.float32) for s in (3000, 3100)]
    sc = sig.scales_for_band(50, 8000, 48, 16000.0)
    with cw.Plan(sc, hop=hop, max_len=n, precision=precision) as plan:
        info = plan.info()
        if hop == 1:
            assert info["spectral_parts"] >= 2, info
        if precision != "fp32":
            assert info["num_direct"] > 0 and info["num_spectral"] > 0, info
        xd = [torch.from_numpy(x).cuda() for x in xs]
        refs = []
        for x in xd:
            r = plan.execute(x)
            plan.sync()
            refs.append(r.clone())
        outs = [torch.full_like(refs[0], -7.0) for _ in range(2)]
        sums = []
        for k in range(12):
            i = k % 2
            plan.execute(xd[i], out=outs[i])
            sums.append(outs[i].sum(dim=(1, 2)))   # stream work right after the execute
        torch.cuda.synchronize()
        for k, s in enumerate(sums):
            assert torch.equal(s, refs[k % 2].sum(dim=(1, 2))), k
        for i in range(2):
            assert torch.equal(outs[i], refs[i]), i
