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


def test_adam_checkpoint_resume_continues_the_uninterrupted_run(tmp_path):
    """The training state saved by adam_fit (taps, ratio, Adam moments, iteration, learning-rate
    scale, losses) resumes exactly: 12 iterations, a restart from a fresh model, then the rest,
    gives the taps, ratio and losses of 30 uninterrupted iterations bit for bit."""
    import torch
    from paper_2409_14489_gb300 import train

    class StandIn(torch.nn.Module):
        def __init__(self):
            super().__init__()
            self.taps = torch.nn.Parameter(torch.tensor([[0.3, -0.2, 0.1]], dtype=torch.float32))
            self.ratio = torch.nn.Parameter(torch.tensor(0.5, dtype=torch.float64))

        def forward(self, x):
            basis = torch.stack([x, x.roll(1, -1), x.roll(-1, -1)], dim=-1)
            return (basis * self.taps[0]).sum(-1) + self.ratio.float() * x ** 2

    g = torch.Generator().manual_seed(7)
    x = torch.randn(4, 16, generator=g)
    target = 0.7 * x + 0.05 * x.roll(1, -1) - 0.2 * x ** 2
    loss_fn = lambda y: torch.mean((y - target) ** 2)          # noqa: E731

    ref = StandIn()
    ref_losses = train.adam_fit(ref, x, loss_fn, iters=30, lr_taps=0.05, lr_ratio=0.02)

    ck = str(tmp_path / "state.npz")
    first = StandIn()
    train.adam_fit(first, x, loss_fn, iters=12, lr_taps=0.05, lr_ratio=0.02, checkpoint=ck,
                   every=4)
    # a fresh process would start from the initial model; the state file carries the rest
    again = StandIn()
    losses = train.adam_fit(again, x, loss_fn, iters=30, lr_taps=0.05, lr_ratio=0.02,
                            checkpoint=ck, every=4)
    assert torch.equal(again.taps.detach(), ref.taps.detach())
    assert float(again.ratio.detach()) == float(ref.ratio.detach())
    assert losses == ref_losses
    import numpy as np
    z = np.load(ck)
    assert int(z["iteration"]) == 30 and len(z["losses"]) == 30
