"""Coefficient optimization on the device (differentiation form): Adam on all per-step taps and
the splitting ratio, post-matched-filter MSE loss, on a noiseless received signal from the
oracle's SSFM channel.  The paper's SSFM-style initialization (centre taps only) is the start."""
import math

import numpy as np
import pytest

from oracle import channel
from synth import configs, signals

pytestmark = pytest.mark.gpu


def test_adam_on_taps_and_ratio_reduces_post_mf_mse():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    from paper_2409_14489_gb300.autograd import CBESSFM
    from paper_2409_14489_gb300.train import PostMFMSE, adam_fit, snr_db_from_mse
    lk = configs.Link(n_spans=5, nf_db=None)
    wl = configs.get_workload("c1_tiny").with_(link=lk)
    sig = wl.signal
    p_dbm, n_real = 6.0, 2
    rx, syms = [], []
    for b in range(n_real):
        tx, s = signals.tx_waveform(wl, p_dbm, seed=40 + b)
        rx.append(channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, lk.n_spans,
                                    sig.sample_rate, steps_per_span=200))
        syms.append(s[0])
    x = torch.from_numpy(np.stack(rx).astype(np.complex64)).cuda()
    n_sb, n_st, ntaps = 3, lk.n_spans, 7
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    taps = signals.ssfm_delta_taps(n_st, n_sb, ntaps, w0)
    link = cbessfm.make_link(lk.beta2, lk.span_length, lk.n_spans, sig.sample_rate)
    model = CBESSFM(link, n_sb, n_st, 0.5, taps, 512, 128)
    loss_fn = PostMFMSE(sig.n_samples, sig.sample_rate, sig.baud, sig.rolloff, np.stack(syms),
                        configs.dbm_to_watt(p_dbm) / 2)
    losses = adam_fit(model, x, loss_fn, iters=200, lr_taps=2e-2, lr_ratio=2e-2)
    assert all(np.isfinite(losses))
    snr0, snr1 = snr_db_from_mse(losses[0]), snr_db_from_mse(min(losses[-10:]))
    assert snr1 > snr0 + 0.5, (snr0, snr1)
    assert 0.0 <= float(model.ratio.detach()) <= 1.0
