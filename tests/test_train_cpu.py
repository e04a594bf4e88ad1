"""The training loss of the differentiation form (train.PostMFMSE: matched filter, one sample
per symbol, mean-phase removal, Sec. III-B and IV-A) on CPU, pinned to the oracle's receiver:
zero back to back, and equal to oracle.evaluate.mse after a phase rotation and additive noise."""
import math

import numpy as np
import pytest

from oracle import evaluate
from synth import configs, signals

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["c1_tiny"])
def test_post_mf_mse_matches_the_oracle_receiver(name):
    from paper_2409_14489_gb300.train import PostMFMSE
    wl = configs.get_workload(name)
    sig = wl.signal
    p_dbm = 2.0
    p_pol = configs.dbm_to_watt(p_dbm) / 2
    tx, syms = signals.tx_waveform(wl, p_dbm, seed=5)
    loss_fn = PostMFMSE(sig.n_samples, sig.sample_rate, sig.baud, sig.rolloff, syms[0][None],
                        p_pol, device="cpu")
    b2b = float(loss_fn(torch.from_numpy(tx.astype(np.complex64))))
    assert b2b < 1e-9
    rng = np.random.default_rng(9)
    noise = 0.05 * math.sqrt(p_pol) * (rng.standard_normal(tx.shape)
                                       + 1j * rng.standard_normal(tx.shape))
    y = (tx * np.exp(1j * 0.7) + noise).astype(np.complex64)
    got = float(loss_fn(torch.from_numpy(y)))
    r = evaluate.receive(y.astype(np.complex128), sig.sample_rate, sig.baud, sig.rolloff, 0.0, p_pol)
    want = evaluate.mse(r, syms[0])
    assert got == pytest.approx(want, rel=1e-4)
