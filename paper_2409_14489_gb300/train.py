"""On-device coefficient optimization with the differentiation form.

The paper selects the taps that minimise the mean square error between transmitted and received
symbols after DBP, matched filtering, 1 sample/symbol and mean-phase removal (Sec. III-B), with an
offline finite-difference solver.  Here the same loss is a torch expression of the DBP output and
its gradient flows through the adjoint kernel, so any torch optimizer trains all per-step taps
and the splitting ratio on the device.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np
import torch


def rrc_amplitude(freq: np.ndarray, baud: float, rolloff: float) -> np.ndarray:
    """Root-raised-cosine amplitude response with unit passband."""
    f = np.abs(freq) / baud
    lo, hi = (1.0 - rolloff) / 2.0, (1.0 + rolloff) / 2.0
    g = (f <= lo).astype(np.float64)
    band = (f > lo) & (f <= hi)
    if rolloff > 0:
        g[band] = np.sqrt(0.5 * (1.0 + np.cos(math.pi / rolloff * (f[band] - lo))))
    return g


class PostMFMSE(torch.nn.Module):
    """MSE after matched filter, decimation to 1 sample/symbol and mean-phase removal.

    ``symbols``: (batch, n_sym, 2) transmitted unit-energy symbols; ``p_pol``: launch power per
    polarization (W) so that the matched-filter output is compared at unit scale; ``device``:
    where the loss runs (the DBP output's device).
    """

    def __init__(self, n_samples: int, sample_rate: float, baud: float, rolloff: float,
                 symbols, p_pol: float, ch_offset: float = 0.0, device="cuda"):
        super().__init__()
        self.sps = int(round(sample_rate / baud))
        freq = np.fft.fftfreq(n_samples, d=1.0 / sample_rate)
        g = rrc_amplitude(freq, baud, rolloff)
        t = np.arange(n_samples) / sample_rate
        self.register_buffer("G", torch.tensor(g, dtype=torch.float32, device=device))
        self.register_buffer("shift", torch.tensor(np.exp(-2j * math.pi * ch_offset * t),
                                                   dtype=torch.complex64, device=device))
        self.register_buffer("x", torch.as_tensor(np.asarray(symbols), dtype=torch.complex64,
                                                  device=device))
        self.scale = 1.0 / math.sqrt(p_pol)

    def forward(self, y):
        if y.dim() == 2:
            y = y[None]
        z = y * self.shift[None, :, None]
        mf = torch.fft.ifft(torch.fft.fft(z, dim=1) * self.G[None, :, None], dim=1)
        r = mf[:, :: self.sps, :] * self.scale
        phi = torch.angle(torch.sum(r * torch.conj(self.x), dim=(1, 2), keepdim=True))
        err = r * torch.exp(-1j * phi) - self.x
        return torch.mean(err.real ** 2 + err.imag ** 2)


def adam_fit(model, x_rx, loss_fn, iters: int = 200, lr_taps: float = 1e-2,
             lr_ratio: float = 1e-2) -> List[float]:
    """Adam on the taps (learning rate relative to their largest magnitude) and the ratio.

    Under torch.distributed each rank passes its own realizations (equal counts); the gradients
    are averaged over ranks in FP64 before every update, so all ranks keep identical taps and the
    update is the one of the whole data set.  The returned losses are the rank's own."""
    from . import distributed
    scale = float(model.taps.detach().abs().max())
    scale = distributed.max_over_ranks(scale)                 # the same learning rate everywhere
    opt = torch.optim.Adam([{"params": [model.taps], "lr": lr_taps * scale},
                            {"params": [model.ratio], "lr": lr_ratio}],
                           betas=(0.9, 0.999))
    losses = []
    for _ in range(iters):
        opt.zero_grad(set_to_none=True)
        loss = loss_fn(model(x_rx))
        loss.backward()
        distributed.average_gradients_([model.taps, model.ratio])
        opt.step()
        losses.append(float(loss.detach()))
    return losses


def snr_db_from_mse(mse: float) -> float:
    return -10.0 * math.log10(mse)
