"""Forward fiber channel in FP64 -- oracle input generator (test infrastructure only).

Symmetric split-step Fourier solution of the Manakov equation (the dual-polarization form of
Eq. (NLSE), Sec. II-C: the nonlinear term uses |u|^2 = |x|^2 + |y|^2) with field attenuation
alpha/2, in physical units (field in sqrt(W)):

    dA/dz = j (beta2/2) d^2A/dt^2 - (alpha/2) A - j gamma |A|^2 A

Each span is followed by an ideal EDFA that restores the span loss, optionally adding ASE noise
(complex Gaussian per sample and polarization, power n_sp h nu (G - 1) R per polarization with
n_sp = NF G / (2 (G - 1))).  The sequence is periodic (circular FFTs).
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

PLANCK = 6.62607015e-34
NU_C = 193.41e12          # Hz, carrier used for the ASE photon energy


def linear_factor(beta2: float, alpha: float, dz: float, freq: np.ndarray) -> np.ndarray:
    """Frequency response of dispersion and loss over dz: exp(-j 2 pi^2 beta2 f^2 dz - alpha dz/2)."""
    return np.exp(-1j * 2.0 * math.pi ** 2 * beta2 * freq ** 2 * dz - 0.5 * alpha * dz)


def propagate(field: np.ndarray, beta2: float, gamma: float, alpha: float, span_length: float,
              n_spans: int, sample_rate: float, steps_per_span: int,
              nf_db: Optional[float] = None, seed: int = 0) -> np.ndarray:
    """Propagate ``field`` (L, 2) through ``n_spans`` spans + EDFAs with the symmetric SSFM."""
    A = np.array(field, dtype=np.complex128, copy=True)
    L = A.shape[0]
    freq = np.fft.fftfreq(L, d=1.0 / sample_rate)
    dz = span_length / steps_per_span
    half = linear_factor(beta2, alpha, dz / 2.0, freq)[:, None]
    # Nonlinear length of one step seen from its midpoint: int_{-dz/2}^{dz/2} exp(-alpha z) dz.
    l_nl = dz if alpha == 0.0 else 2.0 * math.sinh(alpha * dz / 2.0) / alpha
    rng = np.random.default_rng(seed)
    gain = math.exp(alpha * span_length)
    for _ in range(n_spans):
        for _ in range(steps_per_span):
            A = np.fft.ifft(np.fft.fft(A, axis=0) * half, axis=0)
            power = np.abs(A[:, 0]) ** 2 + np.abs(A[:, 1]) ** 2
            A = A * np.exp(-1j * gamma * l_nl * power)[:, None]
            A = np.fft.ifft(np.fft.fft(A, axis=0) * half, axis=0)
        A = A * math.sqrt(gain)
        if nf_db is not None and gain > 1.0:
            nf = 10.0 ** (nf_db / 10.0)
            n_sp = nf * gain / (2.0 * (gain - 1.0))
            var = n_sp * PLANCK * NU_C * (gain - 1.0) * sample_rate
            noise = rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2))
            A = A + math.sqrt(var / 2.0) * noise
    return A
