"""Pins of the oracle's per-step streaming form (mode S: oracle.dbp.dbp_mode_s).

* One block per pass (the blocks cover the whole sequence, no overlap): every pass is an exact
  transform of the periodic sequence and the passes compose to the chain, so mode S equals the
  whole-sequence chain (mode U).
* Shifting the input by whole blocks shifts the output alike.
* Without nonlinearity the passes compose to the closed-form dispersion of the whole link, with
  an error that falls as the overlap grows.
* Mode S needs only one step's memory in its overlap, mode B the whole link's: on a long
  multi-step link with an overlap between the two, mode S stays close to mode U while mode B
  does not.
"""
import math

import numpy as np
import pytest

from oracle import dbp
from synth import signals

RNG = np.random.default_rng(4321)


def _field(L, scale=1.0):
    return scale * (RNG.standard_normal((L, 2)) + 1j * RNG.standard_normal((L, 2))) / math.sqrt(2)


def _bandlimited(L, rate, frac=0.8, scale=1.0):
    """Random field whose spectrum occupies the central `frac` of the band."""
    X = np.fft.fft(_field(L, scale), axis=0)
    f = np.fft.fftfreq(L) * rate
    X[np.abs(f) > frac * rate / 2] = 0
    return np.fft.ifft(X, axis=0)


@pytest.mark.parametrize("n_sb", [1, 2, 3, 5])
def test_single_block_mode_s_equals_whole_sequence(n_sb):
    n_fft, n_st = 32, 3
    L = n_sb * n_fft
    taps = signals.random_taps(2, n_st, n_sb, 5, 0.3, spread=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=64e9 * n_sb, link_length=240e3, n_sb=n_sb,
                        ratio=0.3, taps=taps)
    u = _field(L)
    np.testing.assert_allclose(dbp.dbp_mode_s(u, p, n_fft, 0), dbp.dbp_mode_u(u, p), atol=1e-12)


@pytest.mark.parametrize("n_sb", [2, 3])
def test_mode_s_shift_equivariance_by_whole_blocks(n_sb):
    n_fft, overlap, n_st = 32, 8, 2
    V = n_sb * (n_fft - overlap)
    L = V * 6
    taps = signals.random_taps(3, n_st, n_sb, 5, 0.3, spread=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=64e9 * n_sb, link_length=160e3, n_sb=n_sb,
                        ratio=0.3, taps=taps)
    u = _field(L)
    for shift in (V, 3 * V):
        a = dbp.dbp_mode_s(np.roll(u, shift, axis=0), p, n_fft, overlap)
        b = np.roll(dbp.dbp_mode_s(u, p, n_fft, overlap), shift, axis=0)
        np.testing.assert_allclose(a, b, atol=1e-12)


def test_linear_mode_s_converges_to_closed_form_dispersion():
    n_sb, n_fft, n_st = 3, 256, 4
    rate, Z = 96e9, 320e3
    L = n_sb * 2048
    u = _bandlimited(L, rate)
    taps = np.zeros((n_st, n_sb, n_sb, 5))
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=rate, link_length=Z, n_sb=n_sb, ratio=0.3,
                        taps=taps)
    f = np.fft.fftfreq(L) * rate
    want = np.fft.ifft(np.fft.fft(u, axis=0) *
                       np.exp(1j * 2 * math.pi ** 2 * p.beta2 * Z * f ** 2)[:, None], axis=0)
    errs = []
    for overlap in (32, 64, 128):
        got = dbp.dbp_mode_s(u, p, n_fft, overlap)
        errs.append(np.linalg.norm(got - want) / np.linalg.norm(want))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3


def test_mode_s_needs_only_one_steps_memory():
    """8 steps x 80 km at 96 GS/s with 3 subbands (R' = 32 GS/s): one step's dispersion spans
    about 20 subband samples, the whole link about 160.  With N'_ov = 64 mode S covers the
    step but mode B does not cover the link."""
    n_sb, n_fft, overlap, n_st = 3, 256, 64, 8
    rate = 96e9
    L = n_sb * 2048
    u = _bandlimited(L, rate, scale=0.05)
    taps = signals.random_taps(5, n_st, n_sb, 5, 0.5, spread=0.3)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=rate, link_length=640e3, n_sb=n_sb,
                        ratio=0.3, taps=taps)
    ref = dbp.dbp_mode_u(u, p)
    err = lambda y: np.linalg.norm(y - ref) / np.linalg.norm(ref)
    e_s = err(dbp.dbp_mode_s(u, p, n_fft, overlap))
    e_b = err(dbp.dbp_mode_b(u, p, n_fft, overlap))
    assert e_s < 0.1 * e_b, (e_s, e_b)
    assert e_s < 1e-2, e_s
