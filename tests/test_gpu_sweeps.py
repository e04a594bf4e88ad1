"""Experiment sweeps on a synthetic configuration: the paper's trends at context level (Sec. IV,
Figs. 6-7, and the ESSFM/OSSFM comparison of Sec. III-D), computed with the CUDA chain.

Signal: the C1 model (one 32 GBd DP-16QAM channel at 64 GS/s, 2^12 symbols) over 10 x 80 km at
+6 dBm per channel, no noise, through the oracle's FP64 SSFM channel (100 steps per span).
Receiver: the oracle's matched filter, one sample per symbol and mean-phase removal (Sec. IV-A).
Taps: the analytic coefficients of Sec. II-D (cbessfm.analytic_taps) unless trained.  N' and the
overlap keep N = 512 samples per block with N_ov = 256, which covers the link's dispersion memory
(about 240 samples).

What is checked (the figures' curves need the paper's optimized taps and setup; these are the
trends that hold with analytic taps on this link, found first with the FP64 oracle):
* more DBP steps give a higher SNR, and every DBP beats dispersion compensation (EDC);
* coupled subbands beat the single-band ESSFM at two steps (the paper's motivation);
* 21-tap ESSFM beats the single-tap OSSFM (analytic and trained taps alike);
* the SNR after the CUDA chain is within 0.02 dB of the oracle chain's on the same taps.
The splitting-ratio sweep is reported (its optimum moves with the step count) and checked for the
GPU/oracle agreement only.  Every point goes to $CBESSFM_SWEEP_LOG (JSON lines) when it is set.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import channel, dbp as odbp, evaluate
from synth import configs, signals

from parity_utils import Case, make_plan, run_gpu

pytestmark = pytest.mark.gpu

N_SPANS = 10
P_DBM = 6.0
NTAPS = 21
RHOS = (0.0, 0.12, 0.3, 0.5, 0.7, 1.0)


def _log(**point):
    path = os.environ.get("CBESSFM_SWEEP_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(point) + "\n")


@pytest.fixture(scope="module")
def link_data():
    wl = configs.get_workload("c1_tiny").with_(link=configs.Link(n_spans=N_SPANS, nf_db=None))
    lk, sig = wl.link, wl.signal
    rx, syms = [], []
    for seed in (3, 4, 5):
        tx, s = signals.tx_waveform(wl, P_DBM, seed=seed)
        rx.append(channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, N_SPANS,
                                    sig.sample_rate, steps_per_span=100))
        syms.append(s[0])
    return wl, np.stack(rx), np.stack(syms)


def _snr(wl, out, syms):
    sig = wl.signal
    p_pol = configs.dbm_to_watt(P_DBM) / 2
    y = evaluate.receive(out, sig.sample_rate, sig.baud, sig.rolloff, 0.0, p_pol)
    return evaluate.snr_db(y, syms)


def _taps(wl, n_sb, n_st, ntaps):
    from paper_2409_14489_gb300 import cbessfm
    lk, sig = wl.link, wl.signal
    if n_st == 0:
        return np.zeros((0, n_sb, n_sb, ntaps), dtype=np.float32)
    link = cbessfm.make_link(lk.beta2, lk.span_length, N_SPANS, sig.sample_rate, gamma=lk.gamma,
                             alpha=lk.alpha)
    # the field is in sqrt(W) and each step starts at the launch power: reference power 1
    return cbessfm.analytic_taps(link, n_sb, n_st, 1.0, ntaps, 64,
                                 N_SPANS // n_st).astype(np.float32)


def _case(wl, n_sb, n_st, rho, ntaps):
    lk, sig = wl.link, wl.signal
    return Case(n_sb, 512 // n_sb, 256 // n_sb, n_st, ntaps, rho, sig.n_samples,
                span_length=lk.span_length, n_spans=N_SPANS, sample_rate=sig.sample_rate)


def _gpu_snr(wl, rx, syms, n_sb, n_st, rho, ntaps=NTAPS, taps=None, real=0, label=""):
    case = _case(wl, n_sb, n_st, rho, ntaps)
    w = _taps(wl, n_sb, n_st, ntaps) if taps is None else taps
    out = run_gpu(make_plan(case, w), rx[real:real + 1].astype(np.complex64))[0]
    s = _snr(wl, out, syms[real])
    _log(sweep=label, n_sb=n_sb, n_st=n_st, rho=rho, ntaps=ntaps, snr_db=s)
    return s


def test_snr_grows_with_the_step_count_and_beats_edc(link_data):
    wl, rx, syms = link_data
    snrs = [_gpu_snr(wl, rx, syms, 1, n_st, 0.5, label="steps") for n_st in (0, 1, 2, 5, 10)]
    for a, b in zip(snrs, snrs[1:]):
        assert b > a + 0.2, snrs
    assert snrs[-1] > snrs[0] + 3.0, snrs


def test_coupled_subbands_beat_the_single_band_at_two_steps(link_data):
    wl, rx, syms = link_data
    best = {n_sb: max(_gpu_snr(wl, rx, syms, n_sb, 2, rho, label="subbands")
                      for rho in (0.12, 0.3, 0.5)) for n_sb in (1, 2, 4)}
    assert best[2] > best[1] + 0.4, best
    assert best[4] > best[2] - 0.1, best


@pytest.mark.parametrize("n_st", [2, 5])
def test_essfm_beats_ossfm_with_analytic_taps(link_data, n_st):
    wl, rx, syms = link_data
    ossfm = _gpu_snr(wl, rx, syms, 1, n_st, 0.5, ntaps=1, label="ossfm")
    essfm = _gpu_snr(wl, rx, syms, 1, n_st, 0.5, ntaps=NTAPS, label="essfm")
    assert essfm > ossfm + 0.5, (ossfm, essfm)


@pytest.mark.parametrize("n_st", [2, 10])
def test_ratio_sweep_matches_the_oracle(link_data, n_st):
    """SNR vs the splitting ratio: reported, and within 0.02 dB of the FP64 oracle chain on the
    same (FP32-rounded) taps and input."""
    wl, rx, syms = link_data
    lk, sig = wl.link, wl.signal
    w = _taps(wl, 1, n_st, NTAPS)
    x = rx[0].astype(np.complex64)
    gpu, ref = [], []
    for rho in RHOS:
        gpu.append(_gpu_snr(wl, rx, syms, 1, n_st, rho, taps=w, label="ratio"))
        p = odbp.ChainParams(lk.beta2, sig.sample_rate, lk.span_length * N_SPANS, 1, rho,
                             w.astype(np.float64))
        ref.append(_snr(wl, odbp.dbp_mode_b(x.astype(np.complex128), p, 512, 256), syms[0]))
    assert max(abs(g - r) for g, r in zip(gpu, ref)) <= 0.02, (gpu, ref)
    edc = _gpu_snr(wl, rx, syms, 1, 0, 0.5, label="edc")
    assert min(gpu) > edc, (gpu, edc)


def test_trained_essfm_beats_trained_ossfm(link_data):
    """Adam on the taps and the ratio (differentiation form, post-matched-filter MSE) of a
    two-step ESSFM (21 taps) and OSSFM (1 tap), trained on two realizations and evaluated on a
    third: training does not lose against the analytic start, and ESSFM keeps its lead."""
    import torch
    from paper_2409_14489_gb300 import cbessfm
    from paper_2409_14489_gb300.autograd import CBESSFM
    from paper_2409_14489_gb300.train import PostMFMSE, adam_fit
    wl, rx, syms = link_data
    lk, sig = wl.link, wl.signal
    link = cbessfm.make_link(lk.beta2, lk.span_length, N_SPANS, sig.sample_rate)
    x_train = torch.from_numpy(rx[1:3].astype(np.complex64)).cuda()
    loss_fn = PostMFMSE(sig.n_samples, sig.sample_rate, sig.baud, sig.rolloff, syms[1:3],
                        configs.dbm_to_watt(P_DBM) / 2)
    result = {}
    for ntaps in (1, NTAPS):
        w0 = _taps(wl, 1, 2, ntaps)
        before = _gpu_snr(wl, rx, syms, 1, 2, 0.5, ntaps=ntaps, taps=w0, label="untrained")
        model = CBESSFM(link, 1, 2, 0.5, w0, 512, 256)
        losses = adam_fit(model, x_train, loss_fn, iters=150, lr_taps=1e-2, lr_ratio=1e-2)
        assert all(math.isfinite(v) for v in losses)
        w1 = model.taps.detach().cpu().numpy()
        rho1 = float(model.ratio.detach())
        after = _gpu_snr(wl, rx, syms, 1, 2, rho1, ntaps=ntaps, taps=w1, label="trained")
        result[ntaps] = (before, after, rho1)
        assert after > before - 0.1, result
    assert result[NTAPS][1] > result[1][1] + 0.5, result
