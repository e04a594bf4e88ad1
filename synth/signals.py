"""Seeded signal and coefficient generators (numpy, FP64).

Transmitter model (Sec. IV-A of the paper): uniform square QAM per polarization with unit mean
energy, root-raised-cosine pulses applied in the frequency domain, WDM channels at offsets
``(c - (n_ch - 1) / 2) * spacing``, launch power per channel split equally over the two
polarizations.  The waveform is one period of a periodic sequence (circular filtering).
Field layout everywhere: ``(L, 2)`` complex, sample-major, polarization-minor (x, y), in
sqrt(W).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

from .configs import Workload, dbm_to_watt


def qam_symbols(rng: np.random.Generator, order: int, shape) -> np.ndarray:
    """Uniform square QAM symbols with unit mean energy."""
    m = int(round(math.sqrt(order)))
    assert m * m == order, "square QAM only"
    levels = 2.0 * np.arange(m) - (m - 1)
    norm = math.sqrt(2.0 * (order - 1) / 3.0)
    i = rng.integers(0, m, size=shape)
    q = rng.integers(0, m, size=shape)
    return (levels[i] + 1j * levels[q]) / norm


def rrc_amplitude(freq: np.ndarray, baud: float, rolloff: float) -> np.ndarray:
    """Root-raised-cosine amplitude response with unit passband (G(0) = 1).

    Its square is the raised cosine whose folded spectrum is constant, so a transmit filter
    ``sps * G`` followed by a matched filter ``G`` gives zero ISI at the symbol instants.
    """
    f = np.abs(freq) / baud
    lo = (1.0 - rolloff) / 2.0
    hi = (1.0 + rolloff) / 2.0
    g = np.zeros_like(f)
    g[f <= lo] = 1.0
    band = (f > lo) & (f <= hi)
    if rolloff > 0:
        g[band] = np.sqrt(0.5 * (1.0 + np.cos(math.pi / rolloff * (f[band] - lo))))
    return g


def tx_waveform(wl: Workload, launch_dbm: float, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """Transmitted WDM field of one realization.

    Returns ``(field, symbols)``: field ``(L, 2)`` complex128 in sqrt(W) with average power
    ``n_ch * P_launch``; symbols ``(n_ch, n_sym, 2)`` (unit energy, before power scaling).
    """
    sig = wl.signal
    rng = np.random.default_rng(seed)
    L = sig.n_samples
    sps = sig.sample_rate / sig.baud
    isps = int(round(sps))
    assert abs(sps - isps) < 1e-12, "integer samples per symbol per channel"
    syms = qam_symbols(rng, sig.qam, (sig.n_ch, sig.n_sym, 2))
    freq = np.fft.fftfreq(L, d=1.0 / sig.sample_rate)
    G = rrc_amplitude(freq, sig.baud, sig.rolloff)
    p_pol = dbm_to_watt(launch_dbm) / 2.0
    t = np.arange(L) / sig.sample_rate
    field = np.zeros((L, 2), dtype=np.complex128)
    for c in range(sig.n_ch):
        up = np.zeros((L, 2), dtype=np.complex128)
        up[::isps, :] = syms[c]
        shaped = np.fft.ifft(np.fft.fft(up, axis=0) * (isps * G)[:, None], axis=0)
        fc = (c - (sig.n_ch - 1) / 2.0) * sig.ch_spacing
        field += math.sqrt(p_pol) * shaped * np.exp(2j * math.pi * fc * t)[:, None]
    return field, syms


def effective_length(alpha: float, length: float) -> float:
    """L_eff = (1 - exp(-alpha L)) / alpha (alpha = power attenuation)."""
    if alpha == 0.0:
        return length
    return (1.0 - math.exp(-alpha * length)) / alpha


def ssfm_delta_taps(n_st: int, n_sb: int, ntaps: int, phase_per_step) -> np.ndarray:
    """SSFM-style initial taps: all zero except the centre tap of the SPM and XPM filters.

    ``phase_per_step`` (scalar or length ``n_st``) is the nonlinear phase per unit intensity of
    each step, e.g. gamma * L_eff of the step.  The XPM centre taps carry the 3/2 degeneracy
    factor of the dual-polarization coupled model, so the taps are the effective ones the
    kernel applies.
    """
    phi = np.broadcast_to(np.asarray(phase_per_step, dtype=np.float64), (n_st,))
    w = np.zeros((n_st, n_sb, n_sb, ntaps), dtype=np.float64)
    nc = ntaps // 2
    for s in range(n_st):
        for i in range(n_sb):
            for l in range(n_sb):
                w[s, i, l, nc] = phi[s] * (1.0 if i == l else 1.5)
    return w


def random_taps(seed: int, n_st: int, n_sb: int, ntaps: int, scale: float,
                spread: float = 0.2) -> np.ndarray:
    """SSFM-init taps of size ``scale`` plus a seeded uniform perturbation on every tap.

    Used to stress parity: every tap (including the asymmetric XPM ones) is non-zero.
    """
    rng = np.random.default_rng(seed)
    w = ssfm_delta_taps(n_st, n_sb, ntaps, scale)
    w += scale * spread * rng.uniform(-1.0, 1.0, size=w.shape)
    return w


def batch_jobs_c3(seed: int = 3, n_jobs: int = 256) -> List[dict]:
    """Job list of the batched workload: uneven lengths, step and band counts.

    Lengths are log-uniform from 2^12 to 2^17 symbols (2 samples/symbol, rounded to a
    multiple of 64 samples), steps uniform in {1, 2, 4, 8, 15}, bands in {1, 3, 5}.
    """
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n_jobs):
        n_sym = int(round(2.0 ** rng.uniform(12.0, 17.0)))
        n_samples = max(64, (2 * n_sym) // 64 * 64)
        jobs.append(dict(n_samples=n_samples,
                         n_st=int(rng.choice([1, 2, 4, 8, 15])),
                         n_sb=int(rng.choice([1, 3, 5])),
                         seed=int(seed * 100003 + k)))
    return jobs
