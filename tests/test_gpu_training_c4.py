"""Coefficient optimization at the differentiation workload's scale (Sec. III-B, III-C: the
paper fits the per-step taps offline; here by Adam on the device, through the adjoint kernel).

Workload (c4_adjoint): 32 realizations x 2^15 symbols of the c1 signal model (one DP-16QAM
32 GBd channel, RRC 0.1, 2 samples/symbol) at 0 dBm over 15 x 80 km of noiseless SMF; DBP with
N_sb = 5, N_st = 15, 11 taps per band pair, N' = 1024, N'_ov = 256; all 15 x 25 x 11 taps and the
splitting ratio are trained, 200 Adam iterations of the post-matched-filter MSE, from the
paper's SSFM-style initialization (centre taps gamma L_eff, 3/2 XPM factor) and rho = 0.3.

The received fields come from the oracle's symmetric SSFM channel with 50 steps per span, run
once per session in spawned worker processes (the test process has a CUDA context).  With
CBESSFM_TRAIN_LOG set, the loss curve and the time per iteration are written there as JSON."""
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np
import pytest

from oracle import channel
from synth import configs, signals

pytestmark = pytest.mark.gpu

STEPS_PER_SPAN = 50


def _received(k: int):
    wl = configs.get_workload("c4_adjoint")
    lk, sig = wl.link, wl.signal
    tx, syms = signals.tx_waveform(wl, wl.launch_dbm[k], seed=400 + k)
    rx = channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, lk.n_spans,
                           sig.sample_rate, steps_per_span=STEPS_PER_SPAN)
    return rx.astype(np.complex64), syms[0]


@pytest.fixture(scope="module")
def c4_received():
    wl = configs.get_workload("c4_adjoint")
    n = wl.batch
    workers = max(1, min(n, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        out = pool.map(_received, range(n))
    return wl, np.stack([o[0] for o in out]), np.stack([o[1] for o in out])


def test_c4_scale_adam_training(c4_received):
    import torch
    from paper_2409_14489_gb300 import cbessfm
    from paper_2409_14489_gb300.autograd import CBESSFM
    from paper_2409_14489_gb300.train import PostMFMSE, adam_fit, snr_db_from_mse
    wl, rx, syms = c4_received
    lk, sig, d = wl.link, wl.signal, wl.dbp
    x = torch.from_numpy(rx).cuda()
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    taps = signals.ssfm_delta_taps(d.n_st, d.n_sb, d.ntaps, w0)
    link = cbessfm.make_link(lk.beta2, lk.span_length, lk.n_spans, sig.sample_rate)
    model = CBESSFM(link, d.n_sb, d.n_st, d.ratio, taps, d.n_fft, d.overlap)
    loss_fn = PostMFMSE(sig.n_samples, sig.sample_rate, sig.baud, sig.rolloff, syms,
                        configs.dbm_to_watt(wl.launch_dbm[0]) / 2)
    adam_fit(model, x, loss_fn, iters=2)                    # warm-up (plans, workspaces)
    model = CBESSFM(link, d.n_sb, d.n_st, d.ratio, taps, d.n_fft, d.overlap)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = adam_fit(model, x, loss_fn, iters=200, lr_taps=2e-2, lr_ratio=2e-2)
    torch.cuda.synchronize()
    ms_per_iter = 1e3 * (time.perf_counter() - t0) / 200
    rho = float(model.ratio.detach())
    log = os.environ.get("CBESSFM_TRAIN_LOG")
    if log:
        with open(log, "w") as f:
            json.dump({"workload": "c4_adjoint", "iterations": 200, "ms_per_iteration": ms_per_iter,
                       "rho": rho, "loss": losses,
                       "snr_db": [snr_db_from_mse(v) for v in losses]}, f)
    assert all(np.isfinite(losses))
    # a falling trend: the mean loss of each 20-iteration window below the first window's, the
    # last window the lowest but for noise, and an SNR gain over the SSFM-init start
    win = np.asarray(losses).reshape(10, 20).mean(axis=1)
    assert (win[1:] < win[0]).all(), win
    assert win[-1] <= win.min() * 1.02, win
    snr0, snr1 = snr_db_from_mse(losses[0]), snr_db_from_mse(win[-1])
    assert snr1 > snr0 + 0.2, (snr0, snr1)
    assert 0.0 <= rho <= 1.0
