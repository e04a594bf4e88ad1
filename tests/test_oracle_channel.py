"""Pins of the oracle's forward channel (oracle.channel) and receiver (oracle.evaluate), and the
end-to-end physics check of the DBP chain: a noiseless forward simulation undone by a many-step
DBP recovers the transmitted field.

* gamma = 0: the channel is the closed-form dispersion exp(-j beta2 w^2 Z / 2) (Eq. (GVD_transfer-
  function)); the EDFAs restore the span loss exactly.
* beta2 = 0: the closed-form SPM rotation exp(-j gamma L_eff |A|^2) per span.
* alpha = 0: energy is conserved.
* ASE power per polarization matches n_sp h nu (G - 1) R per span.
* Back-to-back: matched filter + decimation returns the transmitted symbols exactly, for every
  WDM channel (pins the RRC normalization and the channel offsets).
* Forward 1000-step SSFM then CB-ESSFM DBP (one band, centre-tap filters with the per-step
  nonlinear phase gamma * integral of the power profile): error falls with the step count.
"""
import math

import numpy as np
import pytest

from oracle import channel, dbp, evaluate
from synth import configs, signals


def test_linear_channel_is_closed_form_dispersion():
    rng = np.random.default_rng(0)
    L, R = 2048, 64e9
    u = rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2))
    out = channel.propagate(u, beta2=-21.7e-27, gamma=0.0, alpha=4.6e-5, span_length=80e3,
                            n_spans=3, sample_rate=R, steps_per_span=20)
    w = 2 * math.pi * np.fft.fftfreq(L, d=1 / R)
    want = np.fft.ifft(np.fft.fft(u, axis=0) *
                       np.exp(-1j * -21.7e-27 * w ** 2 * 240e3 / 2)[:, None], axis=0)
    assert np.linalg.norm(out - want) / np.linalg.norm(want) < 1e-12


def test_zero_dispersion_channel_is_closed_form_spm():
    rng = np.random.default_rng(1)
    L = 512
    u = 0.05 * (rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2)))
    alpha, Lsp, gamma, ns = 4.6e-5, 80e3, 1.3e-3, 2
    out = channel.propagate(u, beta2=0.0, gamma=gamma, alpha=alpha, span_length=Lsp,
                            n_spans=ns, sample_rate=64e9, steps_per_span=37)
    I = np.abs(u[:, 0]) ** 2 + np.abs(u[:, 1]) ** 2
    leff = (1 - math.exp(-alpha * Lsp)) / alpha
    want = u * np.exp(-1j * gamma * ns * leff * I)[:, None]
    np.testing.assert_allclose(out, want, atol=1e-12)


def test_lossless_channel_conserves_energy():
    wl = configs.get_workload("c1_tiny")
    u, _ = signals.tx_waveform(wl, 6.0, seed=2)
    out = channel.propagate(u, beta2=-21.7e-27, gamma=1.3e-3, alpha=0.0, span_length=80e3,
                            n_spans=1, sample_rate=64e9, steps_per_span=50)
    assert np.sum(np.abs(out) ** 2) == pytest.approx(np.sum(np.abs(u) ** 2), rel=1e-12)


def test_ase_noise_power():
    L, R, ns, nf_db = 1 << 16, 64e9, 4, 5.0
    alpha = configs.Link().alpha
    out = channel.propagate(np.zeros((L, 2), complex), beta2=-21.7e-27, gamma=1.3e-3,
                            alpha=alpha, span_length=80e3, n_spans=ns, sample_rate=R,
                            steps_per_span=4, nf_db=nf_db, seed=9)
    G = math.exp(alpha * 80e3)
    nsp = 10 ** (nf_db / 10) * G / (2 * (G - 1))
    per_pol = nsp * channel.PLANCK * channel.NU_C * (G - 1) * R
    meas = np.mean(np.abs(out) ** 2, axis=0)
    np.testing.assert_allclose(meas, ns * per_pol, rtol=0.03)


@pytest.mark.parametrize("name", ["c1_tiny", "c2_wdm15"])
def test_back_to_back_matched_filter_returns_symbols(name):
    wl = configs.get_workload(name)
    if name == "c2_wdm15":
        wl = wl.with_(signal=configs.Signal(n_ch=5, baud=64e9, ch_spacing=100e9, qam=64,
                                            rolloff=0.05, n_sym=2 ** 10, sample_rate=640e9))
    sig = wl.signal
    p_dbm = 1.0
    tx, syms = signals.tx_waveform(wl, p_dbm, seed=3)
    assert np.mean(np.sum(np.abs(tx) ** 2, axis=1)) == pytest.approx(
        sig.n_ch * configs.dbm_to_watt(p_dbm), rel=0.05)
    for c in range(sig.n_ch):
        fc = (c - (sig.n_ch - 1) / 2) * sig.ch_spacing
        y = evaluate.receive(tx, sig.sample_rate, sig.baud, sig.rolloff, fc,
                             configs.dbm_to_watt(p_dbm) / 2)
        np.testing.assert_allclose(y, syms[c], atol=1e-9)
        assert evaluate.snr_db(y, syms[c]) > 150


def test_snr_of_known_noise_and_phase_removal():
    rng = np.random.default_rng(4)
    x = signals.qam_symbols(rng, 16, (1 << 15, 2))
    sigma2 = 1e-2
    n = math.sqrt(sigma2 / 2) * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
    y = (x + n) * np.exp(0.7j)
    assert evaluate.snr_db(y, x) == pytest.approx(20.0, abs=0.1)


def _per_step_phase(gamma, alpha, span, n_spans, n_st):
    """Nonlinear phase per unit launch power of each DBP step (DBP runs the link backwards)."""
    k = n_st // n_spans
    d = span / k
    fwd = [gamma * math.exp(-alpha * q * d) * (1 - math.exp(-alpha * d)) / alpha
           for _ in range(n_spans) for q in range(k)]
    return np.array(fwd[::-1])


@pytest.mark.slow
def test_forward_then_dbp_recovers_transmitted_field():
    wl = configs.get_workload("c1_tiny")
    lk, sig = wl.link, wl.signal
    p_dbm = 6.0                              # strong nonlinearity so that DBP visibly matters
    tx, syms = signals.tx_waveform(wl, p_dbm, seed=1)
    rx = channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, lk.n_spans,
                           sig.sample_rate, steps_per_span=1000)
    errs = []
    for n_st in (0, 2, 8, 32, 200):
        if n_st == 0:
            taps = np.zeros((0, 1, 1, 1))
        else:
            taps = signals.ssfm_delta_taps(n_st, 1, 1, _per_step_phase(
                lk.gamma, lk.alpha, lk.span_length, lk.n_spans, n_st))
        p = dbp.ChainParams(beta2=lk.beta2, sample_rate=sig.sample_rate,
                            link_length=lk.length, n_sb=1, ratio=0.5, taps=taps)
        out = dbp.dbp_mode_u(rx, p)
        errs.append(np.linalg.norm(out - tx) / np.linalg.norm(tx))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3, errs
    assert errs[0] > 20 * errs[-1], errs      # nonlinear compensation beats dispersion-only
    # and the received symbols improve accordingly
    p_pol = configs.dbm_to_watt(p_dbm) / 2
    y = evaluate.receive(out, sig.sample_rate, sig.baud, sig.rolloff, 0.0, p_pol)
    assert evaluate.snr_db(y, syms[0]) > 50
