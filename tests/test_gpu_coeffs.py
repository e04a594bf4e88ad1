"""Analytic CB-ESSFM coefficients on the GPU (cbessfm_analytic_taps, FP64) against the FP64
oracle (oracle/coeffs.py) on the same quadrature grid, and in use: the CUDA chain with analytic
taps against the oracle chain, and its SNR gain over dispersion compensation."""
import math

import numpy as np
import pytest

from oracle import channel, coeffs as oc, dbp as odbp, evaluate
from synth import configs, signals

from parity_utils import Case, make_plan, oracle_params, rel_l2, run_gpu

pytestmark = pytest.mark.gpu

BETA2 = -21.7e-27
GAMMA = 1.3e-3
ALPHA = 0.2 / (10 * math.log10(math.e)) / 1e3

CASES = [
    # bands, steps, spans_per_step, n_spans, span_length, rate, ntaps, grid, alpha
    (1, 1, 1, 1, 80e3, 64e9, 5, 32, ALPHA),
    (3, 2, 1, 2, 80e3, 192e9, 11, 48, ALPHA),
    (5, 3, 1, 1, 60e3, 640e9, 11, 64, 0.0),           # steps shorter than a span
    (5, 2, 2, 4, 80e3, 320e9, 21, 40, ALPHA),         # two spans per step
    (2, 1, 1, 1, 100e3, 128e9, 63, 63, ALPHA),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"sb{c[0]}_st{c[1]}_nsp{c[2]}_t{c[6]}_M{c[7]}")
def test_analytic_taps_match_oracle(case):
    from paper_2409_14489_gb300 import cbessfm
    bands, steps, nsp, n_spans, lsp, rate, ntaps, grid, alpha = case
    link = cbessfm.make_link(BETA2, lsp, n_spans, rate, gamma=GAMMA, alpha=alpha)
    powers = np.linspace(1.0, 0.5, steps) * 1e-3
    w, resp = cbessfm.analytic_taps(link, bands, steps, powers, ntaps, grid, nsp,
                                    with_response=True)
    L_step = lsp * n_spans / steps
    want = oc.dbp_taps(BETA2, GAMMA, alpha, L_step, nsp, powers, rate, bands, ntaps, grid)
    assert np.max(np.abs(w - want)) <= 1e-12 * np.max(np.abs(want))
    for d in range(-(bands - 1), bands):
        c = oc.coefficients(BETA2, GAMMA, alpha, L_step, nsp, 1.0, rate / bands, d * rate / bands,
                            ntaps, grid)
        assert np.max(np.abs(resp[d + bands - 1] - c)) <= 1e-12 * np.max(np.abs(c))


def test_gpu_chain_with_analytic_taps():
    """C1 signal model over 5 x 80 km at +6 dBm, one step per span, analytic taps: the CUDA chain
    matches the oracle chain and gains over dispersion compensation."""
    from paper_2409_14489_gb300 import cbessfm
    wl = configs.get_workload("c1_tiny")
    lk, sig = wl.link, wl.signal
    n_spans, p_dbm, ntaps = 5, 6.0, 21
    tx, syms = signals.tx_waveform(wl, p_dbm, seed=3)
    rx = channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, n_spans,
                           sig.sample_rate, steps_per_span=200)
    link = cbessfm.make_link(lk.beta2, lk.span_length, n_spans, sig.sample_rate,
                             gamma=lk.gamma, alpha=lk.alpha)
    w = cbessfm.analytic_taps(link, 1, n_spans, 1.0, ntaps, 64)
    case = Case(1, 256, 128, n_spans, ntaps, 0.5, sig.n_samples, span_length=lk.span_length,
                n_spans=n_spans, sample_rate=sig.sample_rate)
    plan = make_plan(case, w)
    got = run_gpu(plan, rx.astype(np.complex64)[None])[0]
    want = odbp.dbp_mode_b(rx.astype(np.complex64).astype(np.complex128),
                           oracle_params(case, w.astype(np.float32).astype(np.float64)),
                           case.n_fft, case.overlap)
    assert rel_l2(got, want, "analytic-taps/c1x5") <= 1e-5
    p_w = configs.dbm_to_watt(p_dbm)
    snr = lambda out: evaluate.snr_db(evaluate.receive(out, sig.sample_rate, sig.baud,
                                                       sig.rolloff, 0.0, p_w / 2), syms[0])
    edc = odbp.dbp_mode_b(rx, odbp.ChainParams(lk.beta2, sig.sample_rate, lk.span_length * n_spans,
                                               1, 0.5, np.zeros((0, 1, 1, ntaps))), 256, 128)
    assert snr(got) > snr(edc) + 2.0
