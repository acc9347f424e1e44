"""Pins for the float64 oracle: each check is fixed by the definition of the
transform (Eq. 1 of the paper discretised with dt = 1 sample, evaluated at
b = k*H per Sec. II.B), not by the oracle's own code.

* closed form: the response to exp(i 2 pi nu n) is exp(i 2 pi nu b) G_a(nu)
  with G_a(nu) = sqrt(a) sum_m exp(-pi^2 B (a(nu - m) - C)^2) (Poisson
  summation of the sampled Gaussian-windowed wavelet), and the scalogram of
  a real cosine is half the modulus of the two such terms at +nu and -nu;
* hop semantics: CWTH(H) is the full transform CWTH(1) kept at every H-th
  sample, bitwise; delaying the input by one hop delays the frames by one,
  bitwise;
* linearity and time reversal (conjugate symmetry of the Morlet taps);
* a pure-Python evaluation of Eq. 1 on tiny inputs (no truncation);
* the truncated sum against the untruncated one;
* numpy's FFT used as a library routine for the same linear convolution,
  with and without folding the spectrum by the hop.

``test_mutants_are_caught`` plants plausible mistakes in copies of the
oracle's C source and checks that these pins reject every one of them.
"""
from __future__ import annotations

import cmath
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from paper_2408_14302_gb300 import signals

B, C = 1.5, 1.0


def poisson_G(a: float, nu: float, bandwidth: float = B, center: float = C) -> float:
    """sqrt(a) * sum_m exp(-pi^2 B (a (nu - m) - C)^2), terms |m| <= 4."""
    return math.sqrt(a) * sum(
        math.exp(-math.pi ** 2 * bandwidth * (a * (nu - m) - center) ** 2)
        for m in range(-4, 5))


# ---------------------------------------------------------------- checks
# Each returns a float error measure so the mutant test can reuse it.

def closed_form_error(cwth_fn, half_support_fn) -> float:
    n = 3000
    worst = 0.0
    for a in (2.0, 2.5, 3.3, 10.0, 40.0):
        h = half_support_fn(a, B)
        for nu in (0.05, 0.2, 0.45, -0.3, -0.45, C / a):
            t = np.arange(n, dtype=np.float64)
            xc = np.cos(2 * np.pi * nu * t)
            xs = np.sin(2 * np.pi * nu * t)
            w = cwth_fn(xc, [a], 1)[0] + 1j * cwth_fn(xs, [a], 1)[0]
            b = np.arange(h, n - h)
            expect = np.exp(2j * np.pi * nu * b) * poisson_G(a, nu)
            err = np.max(np.abs(w[b] - expect)) / max(1.0, poisson_G(a, nu))
            worst = max(worst, float(err))
    return worst


def hop_decimation_mismatch(cwth_fn) -> int:
    x = signals.tones_clip(seed=3, n=2500)
    sc = signals.scales_for_band(100, 8000, 6, 16000.0)
    w1 = cwth_fn(x, sc, 1)
    bad = 0
    for hop in (3, 64, 128, 700):
        wh = cwth_fn(x, sc, hop)
        bad += int(not np.array_equal(wh, w1[:, ::hop]))
    return bad


def shift_mismatch(cwth_fn) -> int:
    x = signals.tones_clip(seed=4, n=2000)
    sc = signals.scales_for_band(100, 8000, 5, 16000.0)
    bad = 0
    for hop in (1, 16, 100):
        w = cwth_fn(x, sc, hop)
        xs = np.concatenate([np.zeros(hop), x])
        ws = cwth_fn(xs, sc, hop)
        bad += int(ws.shape[1] != w.shape[1] + 1)
        bad += int(not np.array_equal(ws[:, 1:], w))
    return bad


def reversal_error(cwth_fn) -> float:
    x = signals.tones_clip(seed=5, n=1500)
    sc = [2.0, 7.5, 31.0]
    w = cwth_fn(x, sc, 1)
    wr = cwth_fn(x[::-1].copy(), sc, 1)
    return float(np.max(np.abs(wr - np.conj(w[:, ::-1]))) / np.max(np.abs(w)))


def brute_force_error(cwth_fn_untrunc) -> float:
    """Eq. 1 with dt = 1, evaluated term by term in pure Python."""
    rng = np.random.default_rng(11)
    n, hop = 37, 4
    x = rng.standard_normal(n)
    scales = [2.0, 3.7, 9.0]
    got = cwth_fn_untrunc(x, scales, hop)
    worst = 0.0
    for si, a in enumerate(scales):
        for k in range(-(-n // hop)):
            b = k * hop
            acc = 0j
            for i in range(n):
                u = (i - b) / a
                psi = (math.pi * B) ** -0.5 * math.exp(-u * u / B) * cmath.exp(2j * math.pi * C * u)
                acc += x[i] * psi.conjugate()
            acc /= math.sqrt(a)
            worst = max(worst, abs(got[si, k] - acc) / max(1.0, abs(acc)))
    return worst


def fft_reference(x: np.ndarray, scales, hop: int, fold: bool) -> np.ndarray:
    """Same linear convolution through numpy's FFT.

    The taps g[t] = a^{-1/2} conj(psi(t/a)) act as a correlation whose DTFT,
    by Poisson summation, is sqrt(a) sum_m Psi(a (nu - m)) with
    Psi(f) = exp(-pi^2 B (f - C)^2).  With M >= N + 2*support the circular
    convolution equals the linear one.  With ``fold`` the spectrum is summed
    over the H aliases of each bin r (q = r + jP, P = M/H) and a length-P
    inverse FFT gives the frames directly.
    """
    n = x.shape[0]
    h = int(math.ceil(max(scales) * math.sqrt(B * math.log(1e16))))
    M = hop * int(math.ceil((n + 2 * h) / hop))
    X = np.fft.fft(x, M)
    nu = np.arange(M) / M
    out = []
    for a in scales:
        G = sum(np.exp(-np.pi ** 2 * B * (a * (nu - m) - C) ** 2) for m in range(-4, 5))
        Y = X * (math.sqrt(a) * G)
        if fold:
            P = M // hop
            Z = Y.reshape(hop, P).sum(axis=0)
            w = np.fft.ifft(Z) / hop
        else:
            w = np.fft.ifft(Y)[::hop]
        out.append(w[: -(-n // hop)])
    return np.array(out)


def fft_error(cwth_fn) -> float:
    x = signals.tones_clip(seed=6, n=4000)
    sc = signals.scales_for_band(100, 8000, 8, 16000.0)
    worst = 0.0
    for hop in (1, 32, 64):
        w = cwth_fn(x, sc, hop)
        for fold in (False, True):
            if fold and hop == 1:
                continue
            ref = fft_reference(x, sc, hop, fold)
            worst = max(worst, float(np.max(np.abs(w - ref)) / np.max(np.abs(ref))))
    return worst


# ---------------------------------------------------------------- tests

def test_closed_form_complex_exponential(oracle_mod):
    assert closed_form_error(oracle_mod.cwth, oracle_mod.half_support) < 1e-12


def test_closed_form_real_cosine_magnitude(oracle_mod):
    # cos(2 pi nu n) = (e^{i 2 pi nu n} + e^{-i 2 pi nu n}) / 2, so at interior
    # frames |W(b)| = |e^{i 2 pi nu b} G_a(nu) + e^{-i 2 pi nu b} G_a(-nu)| / 2:
    # the scalogram itself (cwth_magnitude) against the two-term closed form.
    n = 2000
    t = np.arange(n, dtype=np.float64)
    for a, nu in ((2.0, 0.3), (4.0, 0.25), (12.0, 0.08), (30.0, 0.02)):
        h = oracle_mod.half_support(a, B)
        mag = oracle_mod.cwth_magnitude(np.cos(2 * np.pi * nu * t), [a], 1)[0]
        b = np.arange(h, n - h)
        expect = np.abs(np.exp(2j * np.pi * nu * b) * poisson_G(a, nu)
                        + np.exp(-2j * np.pi * nu * b) * poisson_G(a, -nu)) / 2
        assert np.max(np.abs(mag[b] - expect)) <= 1e-12 * max(1.0, float(np.max(expect)))


def test_alias_term_matters_at_small_scale():
    # At a = 2 the m = -1 alias carries the response to nu = -0.45; a
    # single-lobe spectrum would predict ~0 there.
    assert poisson_G(2.0, -0.45) > 1.0
    single = math.sqrt(2.0) * math.exp(-math.pi ** 2 * B * (2.0 * -0.45 - C) ** 2)
    assert single < 1e-20


def test_hop_is_bitwise_decimation(oracle_mod):
    assert hop_decimation_mismatch(oracle_mod.cwth) == 0


def test_shift_by_one_hop_is_bitwise(oracle_mod):
    assert shift_mismatch(oracle_mod.cwth) == 0


def test_linearity(oracle_mod):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(1200)
    y = signals.tones_clip(seed=8, n=1200)
    sc = [2.0, 5.0, 20.0]
    w = oracle_mod.cwth(2.5 * x - 0.75 * y, sc, 8)
    ref = 2.5 * oracle_mod.cwth(x, sc, 8) - 0.75 * oracle_mod.cwth(y, sc, 8)
    assert np.max(np.abs(w - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_time_reversal_conjugates(oracle_mod):
    assert reversal_error(oracle_mod.cwth) < 1e-13


def test_brute_force_eq1_tiny(oracle_mod):
    fn = lambda x, s, h: oracle_mod.cwth(x, s, h, truncate=False)
    assert brute_force_error(fn) < 1e-13


def test_truncation_is_below_eps(oracle_mod):
    x = signals.tones_clip(seed=9, n=1800)
    sc = [2.0, 13.0, 60.0]
    full = oracle_mod.cwth(x, sc, 5, truncate=False)
    trunc = oracle_mod.cwth(x, sc, 5)
    assert np.max(np.abs(full - trunc)) <= 1e-13 * np.max(np.abs(full))


def test_numpy_fft_evaluation_agrees(oracle_mod):
    assert fft_error(oracle_mod.cwth) < 1e-12


def test_frames_and_support(oracle_mod):
    assert oracle_mod.num_frames(16000, 64) == 250
    assert oracle_mod.num_frames(16001, 64) == 251
    assert oracle_mod.num_frames(1, 512) == 1
    # h = ceil(a sqrt(B ln 1e16)) = ceil(7.4338 a)
    assert oracle_mod.half_support(2.0, 1.5) == math.ceil(2.0 * math.sqrt(1.5 * math.log(1e16)))
    assert oracle_mod.half_support(160.0, 1.5) == 1190


def test_rejects_bad_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.cwth(np.ones(10), [0.0], 1)
    with pytest.raises(ValueError):
        oracle_mod.cwth(np.ones(10), [2.0], 0)
    with pytest.raises(ValueError):
        oracle_mod.cwth(np.ones(10), [float("nan")], 1)


# ---------------------------------------------------------------- mutants

MUTANTS = {
    "no_conjugate": ("gim[t + h] = -env * sin(ph);", "gim[t + h] = env * sin(ph);"),
    "no_scale_norm": ("const double norm = 1.0 / sqrt(a) / sqrt(ORACLE_PI * bandwidth);",
                      "const double norm = 1.0 / sqrt(ORACLE_PI * bandwidth);"),
    "gauss_2B": ("exp(-(u * u) / bandwidth)", "exp(-(u * u) / (2.0 * bandwidth))"),
    "shift_sign": ("const double xv = x[b + t];", "const double xv = x[b - t];"),
    "half_freq": ("const double ph = 2.0 * ORACLE_PI * center * u;",
                  "const double ph = ORACLE_PI * center * u;"),
    "short_support": ("return (int64_t)ceil(a * sqrt(bandwidth * log(1.0 / eps)));",
                      "return (int64_t)ceil(0.5 * a * sqrt(bandwidth * log(1.0 / eps)));"),
    "drop_last_tap": ("for (int64_t t = t0; t <= t1; ++t) {", "for (int64_t t = t0; t < t1; ++t) {"),
    "frame_stride": ("const int64_t b = k * (int64_t)hop;", "const int64_t b = k * (int64_t)hop + (k > 0);"),
}


def _build_mutant(src_text: str, tmpdir: str, name: str):
    path = os.path.join(tmpdir, f"{name}.c")
    with open(path, "w") as f:
        f.write(src_text)
    so = os.path.join(tmpdir, f"lib{name}.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", path, "-o", so, "-lm"], check=True)
    lib = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_cwth.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, dp,
                                ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_int32, ctypes.c_int32, dp, dp, dp]
    lib.oracle_half_support.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.oracle_half_support.restype = ctypes.c_int64

    def cwth(x, scales, hop, truncate=True):
        x = np.ascontiguousarray(np.asarray(x, np.float64))
        sc = np.ascontiguousarray(np.asarray(scales, np.float64))
        F = -(-x.shape[0] // hop)
        re = np.empty((sc.shape[0], F)); im = np.empty((sc.shape[0], F))
        rc = lib.oracle_cwth(x.ctypes.data_as(dp), x.shape[0], B, C, sc.ctypes.data_as(dp),
                             sc.shape[0], hop, 1e-16, 1 if truncate else 0, 0,
                             re.ctypes.data_as(dp), im.ctypes.data_as(dp), dp())
        assert rc == 0
        return re + 1j * im

    def half_support(a, bw):
        return int(lib.oracle_half_support(a, bw, 1e-16))

    return cwth, half_support


def _pins_reject(cwth, half_support) -> list[str]:
    failed = []
    if not closed_form_error(cwth, half_support) < 1e-12:
        failed.append("closed_form")
    if hop_decimation_mismatch(cwth) != 0:
        failed.append("hop")
    if shift_mismatch(cwth) != 0:
        failed.append("shift")
    if not reversal_error(cwth) < 1e-13:
        failed.append("reversal")
    if not brute_force_error(lambda x, s, h: cwth(x, s, h, truncate=False)) < 1e-13:
        failed.append("brute")
    if not fft_error(cwth) < 1e-12:
        failed.append("fft")
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants_are_caught(name, tmp_path, oracle_mod):
    src_path = os.path.join(os.path.dirname(oracle_mod.__file__), "cwth_oracle.c")
    src = open(src_path).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    cwth, hs = _build_mutant(src.replace(old, new), str(tmp_path), name)
    assert _pins_reject(cwth, hs), f"mutant {name} passed every pin"


# ---------------------------------------------------------------- resample-first reading
# oracle.cwth_resampled(x, a, H) re-samples y[m] = x[m H] and evaluates Eq. 1
# at every sample of y with scale a / H (paper Sec. III.B, Fig. 2).

def test_resampled_at_hop_1_is_the_cwt(oracle_mod):
    x = signals.tones_clip(seed=11, n=1500)
    sc = signals.scales_for_band(100, 8000, 6, 16000.0)
    assert np.array_equal(oracle_mod.cwth_resampled(x, sc, 1), oracle_mod.cwth(x, sc, 1))


def test_resampled_closed_form(oracle_mod):
    # Re-sampling exp(i 2 pi nu n) at spacing H gives exp(i 2 pi (nu H) m);
    # at interior frames its response at scale a / H is
    # exp(i 2 pi nu H m) sqrt(a/H) sum_k exp(-pi^2 B ((a/H)(nu H - k) - C)^2).
    n, worst = 6000, 0.0
    for H in (3, 8):
        for a in (8.0, 20.0, 64.0):
            ap = a / H
            h = oracle_mod.half_support(ap, B)
            for nu in (0.01, 0.03, -0.02, C / a):
                t = np.arange(n, dtype=np.float64)
                w = (oracle_mod.cwth_resampled(np.cos(2 * np.pi * nu * t), [a], H)[0]
                     + 1j * oracle_mod.cwth_resampled(np.sin(2 * np.pi * nu * t), [a], H)[0])
                m = np.arange(h, len(w) - h)
                g = poisson_G(ap, nu * H)
                expect = np.exp(2j * np.pi * nu * H * m) * g
                worst = max(worst, float(np.max(np.abs(w[m] - expect)) / max(1.0, g)))
    assert worst < 1e-12


def test_resampled_brute_force_tiny(oracle_mod):
    rng = np.random.default_rng(12)
    x = rng.standard_normal(37)
    H, scales = 3, [2.5, 6.0]
    got = oracle_mod.cwth_resampled(x, scales, H, truncate=False)
    y = x[::H]
    for s, a in enumerate(scales):
        ap = a / H
        for m in range(len(y)):
            acc = 0j
            for j in range(len(y)):
                u = (j - m) / ap
                psi = (math.pi * B) ** -0.5 * math.exp(-u * u / B) * complex(
                    math.cos(2 * math.pi * C * u), math.sin(2 * math.pi * C * u))
                acc += y[j] * psi.conjugate()
            assert abs(got[s, m] - acc / math.sqrt(ap)) < 1e-13
