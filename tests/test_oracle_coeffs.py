"""Pins of the analytic-coefficient oracle (oracle/coeffs.py, Sec. II-D of the paper).

* The closed-form kernel (Eq. kernel_analytic) against an independent quadrature of its
  definition (Eq. kernel_definition) for one and several spans, with and without loss.
* Without dispersion every frequency pair sees the same kernel, so the impulse response is a
  single tap: c[m] = P gamma N_sp L_eff delta[m].
* A sum of c[m] over one full period of the grid picks out the kernel's diagonal, where b = 0:
  it equals P gamma N_sp L_eff for any dispersion and subband separation.
* The symmetries the paper states: c_il[m] = c_li[-m] and the even SPM response.
* A lossless step gives a real SPM response (a symmetry of the square domain).
* The midpoint rule converges to the double integral at second order.
* DBP taps: equal for equal l - i, 3/2 factor on XPM, proportional to the step power.
* Physics: backpropagation with analytic taps beats dispersion compensation alone on a channel
  with strong Kerr nonlinearity.
"""
import math

import numpy as np
import pytest

from oracle import channel, coeffs as oc, dbp as odbp, evaluate
from synth import configs, signals

BETA2 = -21.7e-27
GAMMA = 1.3e-3
ALPHA = 0.2 / (10 * math.log10(math.e)) / 1e3      # 0.2 dB/km in 1/m


def leff(alpha, L):
    return (1 - math.exp(-alpha * L)) / alpha if alpha > 0 else L


@pytest.mark.parametrize("n_spans", [1, 2, 3])
@pytest.mark.parametrize("alpha", [ALPHA, 0.0])
def test_closed_form_kernel_matches_its_definition(n_spans, alpha):
    rng = np.random.default_rng(n_spans)
    mu = rng.uniform(-80e9, 80e9, 40)
    nu = rng.uniform(-80e9, 80e9, 40)
    L = 60e3 * n_spans
    a = oc.kernel_closed_form(mu, nu, BETA2, GAMMA, alpha, L, n_spans)
    b = oc.kernel_numeric(mu, nu, BETA2, GAMMA, alpha, L, n_spans, nodes=200)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_kernel_limits_on_the_diagonal():
    # b = 0 on mu = nu (and nu = 0): K = gamma N_sp L_eff,span
    f = np.array([0.0, 10e9, -33e9])
    for n_spans in (1, 4):
        K = oc.kernel_closed_form(f, f, BETA2, GAMMA, ALPHA, 80e3 * n_spans, n_spans)
        assert np.allclose(K, GAMMA * n_spans * leff(ALPHA, 80e3), rtol=1e-13, atol=0)
    K0 = oc.kernel_closed_form(f, f, BETA2, GAMMA, 0.0, 50e3, 1)
    assert np.allclose(K0, GAMMA * 50e3, rtol=1e-13, atol=0)


def test_no_dispersion_gives_a_single_tap():
    P = 2e-3
    for f_sep in (0.0, 12.8e9):
        c = oc.coefficients(0.0, GAMMA, ALPHA, 80e3, 1, P, 12.8e9, f_sep, 11, 32)
        want = np.zeros(11)
        want[5] = P * GAMMA * leff(ALPHA, 80e3)
        assert np.allclose(c, want, rtol=0, atol=1e-15 * want[5])


@pytest.mark.parametrize("f_sep", [0.0, 12.8e9, -25.6e9])
def test_full_period_sum_is_the_nonlinear_phase_of_a_constant_intensity(f_sep):
    P, M = 1e-3, 63
    for n_spans in (1, 2):
        c = oc.coefficients(BETA2, GAMMA, ALPHA, 80e3 * n_spans, n_spans, P, 12.8e9, f_sep, M, M)
        assert abs(np.sum(c) - P * GAMMA * n_spans * leff(ALPHA, 80e3)) <= 1e-12 * abs(np.sum(c))


def test_time_reversal_and_spm_symmetry():
    Rs = 12.8e9
    for f in (0.0, Rs, 2 * Rs):
        c = oc.coefficients(BETA2, GAMMA, ALPHA, 80e3, 1, 1e-3, Rs, f, 11, 48)
        cr = oc.coefficients(BETA2, GAMMA, ALPHA, 80e3, 1, 1e-3, Rs, -f, 11, 48)
        assert np.max(np.abs(c - cr[::-1])) <= 1e-12 * np.max(np.abs(c))     # c_il[m] = c_li[-m]
    c0 = oc.coefficients(BETA2, GAMMA, ALPHA, 80e3, 1, 1e-3, Rs, 0.0, 11, 48)
    assert np.max(np.abs(c0 - c0[::-1])) <= 1e-12 * np.max(np.abs(c0))


def test_lossless_spm_response_is_real():
    # alpha = 0 makes K even in b and, on the square centred at 0, mapping (mu, nu) to
    # (-nu, -mu) turns the integral into its own conjugate; loss or a subband offset breaks it
    c = oc.coefficients(BETA2, GAMMA, 0.0, 80e3, 1, 1e-3, 12.8e9, 0.0, 11, 48)
    assert np.max(np.abs(c.imag)) <= 1e-12 * np.max(np.abs(c.real))
    for alpha, f_sep in ((ALPHA, 0.0), (0.0, 12.8e9)):
        c2 = oc.coefficients(BETA2, GAMMA, alpha, 80e3, 1, 1e-3, 12.8e9, f_sep, 11, 48)
        assert np.max(np.abs(c2.imag)) > 1e-3 * np.max(np.abs(c2.real))


def test_midpoint_rule_converges_at_second_order():
    args = (BETA2, GAMMA, ALPHA, 80e3, 1, 1e-3, 12.8e9, 12.8e9, 11)
    c = {M: oc.coefficients(*args, M) for M in (32, 64, 128, 256)}
    d1 = np.max(np.abs(c[64] - c[32]))
    d2 = np.max(np.abs(c[128] - c[64]))
    d3 = np.max(np.abs(c[256] - c[128]))
    assert 3.0 < d1 / d2 < 5.0 and 3.0 < d2 / d3 < 5.0


def test_dbp_taps_structure():
    powers = np.array([1e-3, 0.5e-3, 2e-3])
    w = oc.dbp_taps(BETA2, GAMMA, ALPHA, 40e3, 1, powers, 64e9, 4, 7, 32)
    assert w.shape == (3, 4, 4, 7)
    for s in range(3):
        for d in range(-3, 4):
            pairs = [(i, i + d) for i in range(4) if 0 <= i + d < 4]
            for (i, l) in pairs[1:]:
                assert np.array_equal(w[s, i, l], w[s, pairs[0][0], pairs[0][1]])
    c01 = oc.coefficients(BETA2, GAMMA, ALPHA, 40e3, 1, 1e-3, 16e9, 16e9, 7, 32)
    assert np.allclose(w[0, 0, 1], 1.5 * c01.real, rtol=1e-15, atol=0)
    assert np.allclose(w[1], 0.5 * w[0], rtol=1e-14, atol=0)
    assert np.allclose(w[2], 2.0 * w[0], rtol=1e-14, atol=0)


def test_analytic_taps_beat_dispersion_compensation_on_a_nonlinear_link():
    """Single-channel C1 signal model over 5 x 80 km at +6 dBm (strong Kerr effect): one CB-ESSFM
    step per span with analytic taps (3 subbands) recovers a clearly higher SNR than EDC."""
    wl = configs.get_workload("c1_tiny")
    lk, sig = wl.link, wl.signal
    n_spans, p_dbm = 5, 6.0
    tx, syms = signals.tx_waveform(wl, p_dbm, seed=3)
    rx = channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, n_spans,
                           sig.sample_rate, steps_per_span=200)
    L = lk.span_length * n_spans
    p_w = configs.dbm_to_watt(p_dbm)
    n_fft, overlap, n_sb, ntaps = 256, 128, 1, 21

    def snr_of(out):
        y = evaluate.receive(out, sig.sample_rate, sig.baud, sig.rolloff, 0.0, p_w / 2)
        return evaluate.snr_db(y, syms[0])

    edc = odbp.dbp_mode_b(rx, odbp.ChainParams(lk.beta2, sig.sample_rate, L, n_sb, 0.5,
                                               np.zeros((0, n_sb, n_sb, ntaps))), n_fft, overlap)
    # the waveform is in sqrt(W) and every step starts a span at the launch power, so the taps
    # act on |u|^2 directly: reference power 1 in the units of u
    w = oc.dbp_taps(lk.beta2, lk.gamma, lk.alpha, lk.span_length, 1, np.ones(n_spans),
                    sig.sample_rate, n_sb, ntaps, 64)
    ess = odbp.dbp_mode_b(rx, odbp.ChainParams(lk.beta2, sig.sample_rate, L, n_sb, 0.5, w),
                          n_fft, overlap)
    s_edc, s_ess = snr_of(edc), snr_of(ess)
    assert s_ess > s_edc + 2.0, (s_edc, s_ess)
