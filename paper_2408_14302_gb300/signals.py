"""Seeded synthetic workloads for the hop-size CWT.

This module only draws signals and scale lists; it holds none of the
transform's arithmetic and is the one module that both the CUDA path's tests
and the float64 oracle's tests take their inputs from.

The paper measures on MIMII machine sounds (Sec. III.A: 10 s clips at 16 kHz,
fan/pump/slider/valve, mixed with factory noise at -6/0/6 dB SNR).  That data
set is not available here, so these generators stand in for it:

* ``tones_clip``  - three sinusoids (440, 1200, 3100 Hz; amplitudes 1, 0.5,
  0.25; random phases) plus white Gaussian noise at a given SNR.
* ``machine_clip`` - a machine-like harmonic stack (fundamental uniform in
  20-200 Hz, 10 harmonics with amplitude 1/k, a slow random 1 % frequency
  wobble) plus AR(1)-coloured noise (coefficient 0.9) at an SNR drawn from
  {-6, 0, 6} dB.

SNR is 10 log10(mean(clean^2) / mean(noise^2)) over the clip; the noise is
scaled to hit it exactly.
"""
from __future__ import annotations

import numpy as np

SNR_CHOICES_DB = (-6.0, 0.0, 6.0)


def _scale_noise(clean: np.ndarray, noise: np.ndarray, snr_db: float) -> np.ndarray:
    p_clean = float(np.mean(clean * clean))
    p_noise = float(np.mean(noise * noise))
    if p_noise == 0.0:
        return noise
    gain = np.sqrt(p_clean / (p_noise * 10.0 ** (snr_db / 10.0)))
    return noise * gain


def tones_clip(seed: int = 0, n: int = 16000, fs: float = 16000.0,
               snr_db: float = 6.0, dtype=np.float64) -> np.ndarray:
    """Three tones + white Gaussian noise.  Draw order: 3 phases, then n normals."""
    rng = np.random.default_rng(seed)
    phases = rng.uniform(0.0, 2.0 * np.pi, 3)
    noise = rng.standard_normal(n)
    t = np.arange(n, dtype=np.float64) / fs
    clean = (1.0 * np.sin(2 * np.pi * 440.0 * t + phases[0])
             + 0.5 * np.sin(2 * np.pi * 1200.0 * t + phases[1])
             + 0.25 * np.sin(2 * np.pi * 3100.0 * t + phases[2]))
    x = clean + _scale_noise(clean, noise, snr_db)
    return x.astype(dtype)


def _ar1(u: np.ndarray, coef: float) -> np.ndarray:
    from scipy.signal import lfilter
    return lfilter([1.0], [1.0, -coef], u)


def machine_clip(seed: int, n: int = 160000, fs: float = 16000.0,
                 dtype=np.float32, snr_db: float | None = None) -> np.ndarray:
    """Harmonic stack with a slow 1 % wobble + AR(1) noise.

    Draw order: f0 ~ U(20, 200); wobble knots ~ U(-1, 1) every 0.5 s; 10
    initial phases ~ U(0, 2 pi); n standard normals for the noise drive; the
    SNR from {-6, 0, 6} dB (unless ``snr_db`` is given).
    """
    rng = np.random.default_rng(seed)
    f0 = rng.uniform(20.0, 200.0)
    knot_step = int(round(0.5 * fs))
    n_knots = n // knot_step + 2
    knots = rng.uniform(-1.0, 1.0, n_knots)
    phi0 = rng.uniform(0.0, 2.0 * np.pi, 10)
    u = rng.standard_normal(n)
    snr = float(rng.choice(SNR_CHOICES_DB)) if snr_db is None else float(snr_db)

    idx = np.arange(n, dtype=np.float64)
    wobble = np.interp(idx, np.arange(n_knots) * knot_step, knots)
    inst_f = f0 * (1.0 + 0.01 * wobble)
    phase = 2.0 * np.pi * np.cumsum(inst_f) / fs
    clean = np.zeros(n, dtype=np.float64)
    for k in range(1, 11):
        clean += np.sin(k * phase + phi0[k - 1]) / k
    noise = _ar1(u, 0.9)
    x = clean + _scale_noise(clean, noise, snr)
    return x.astype(dtype)


def machine_batch(n_clips: int, n: int = 160000, fs: float = 16000.0,
                  seed0: int = 1000, dtype=np.float32) -> np.ndarray:
    """[n_clips, n] batch; clip i uses seed seed0 + i."""
    return np.stack([machine_clip(seed0 + i, n, fs, dtype) for i in range(n_clips)])


def geometric_freqs(f_lo: float, f_hi: float, S: int) -> np.ndarray:
    """S frequencies from f_hi down to f_lo, geometrically spaced (both ends in)."""
    if S == 1:
        return np.array([f_hi], dtype=np.float64)
    s = np.arange(S, dtype=np.float64)
    return f_hi * (f_lo / f_hi) ** (s / (S - 1))


def scales_for_band(f_lo: float, f_hi: float, S: int, fs: float,
                    center: float = 1.0) -> np.ndarray:
    """Scales in samples, a_s = C * fs / f_s, ascending (row 0 is f_hi)."""
    return center * fs / geometric_freqs(f_lo, f_hi, S)


# Named workloads (sizes of the paper's setting: 10 s clips at 16 kHz, Sec. III.A).
WORKLOADS = {
    "tones_1s_32scales": dict(n=16000, fs=16000.0, S=32, f_lo=100.0, f_hi=8000.0,
                              hops=(1, 64)),
    "machine_10s_64clips_64scales": dict(n=160000, fs=16000.0, S=64, f_lo=50.0,
                                         f_hi=8000.0, clips=64, hops=(256, 1)),
    "tones_1s_128scales": dict(n=16000, fs=16000.0, S=128, f_lo=100.0, f_hi=8000.0,
                               hops=(64, 128, 256, 512)),
}
