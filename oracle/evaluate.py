"""Receiver-side evaluation in FP64 -- oracle (test infrastructure only).

Sec. IV-A: after DBP, the channel under test is matched-filtered, resampled at one sample per
symbol, its mean phase rotation is removed, and the SNR is the transmitted-symbol power over the
power of the difference between output samples and transmitted symbols.
"""
from __future__ import annotations

import math

import numpy as np


def rrc_response(freq: np.ndarray, baud: float, rolloff: float) -> np.ndarray:
    """Root-raised-cosine amplitude with unit passband; its square is the raised cosine."""
    f = np.abs(freq) / baud
    lo, hi = (1.0 - rolloff) / 2.0, (1.0 + rolloff) / 2.0
    g = np.where(f <= lo, 1.0, 0.0)
    band = (f > lo) & (f <= hi)
    if rolloff > 0:
        g = np.where(band, np.sqrt(0.5 * (1.0 + np.cos(math.pi / rolloff *
                                                         np.clip(f - lo, 0.0, None)))), g)
    return g


def receive(field: np.ndarray, sample_rate: float, baud: float, rolloff: float,
            ch_offset: float, p_pol: float) -> np.ndarray:
    """Matched filter + 1 sample/symbol for the channel at ``ch_offset`` Hz.

    Returns (n_sym, 2) symbol estimates divided by sqrt(p_pol), so a back-to-back link returns the
    transmitted unit-energy symbols exactly.
    """
    L = field.shape[0]
    sps = int(round(sample_rate / baud))
    t = np.arange(L) / sample_rate
    base = field * np.exp(-2j * math.pi * ch_offset * t)[:, None]
    freq = np.fft.fftfreq(L, d=1.0 / sample_rate)
    G = rrc_response(freq, baud, rolloff)
    mf = np.fft.ifft(np.fft.fft(base, axis=0) * G[:, None], axis=0)
    return mf[::sps, :] / math.sqrt(p_pol)


def snr_db(y: np.ndarray, x: np.ndarray) -> float:
    """SNR after removing the mean phase rotation (one phase for both polarizations)."""
    phi = np.angle(np.sum(y * np.conj(x)))
    err = y * np.exp(-1j * phi) - x
    return 10.0 * math.log10(np.sum(np.abs(x) ** 2) / np.sum(np.abs(err) ** 2))


def mse(y: np.ndarray, x: np.ndarray) -> float:
    """Mean square error after mean-phase removal (the loss minimised in Sec. III-B)."""
    phi = np.angle(np.sum(y * np.conj(x)))
    return float(np.mean(np.abs(y * np.exp(-1j * phi) - x) ** 2))
