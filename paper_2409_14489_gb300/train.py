"""On-device coefficient optimization with the differentiation form.

The paper selects the taps that minimise the mean square error between transmitted and received
symbols after DBP, matched filtering, 1 sample/symbol and mean-phase removal (Sec. III-B), with an
offline finite-difference solver.  Here the same loss is a torch expression of the DBP output and
its gradient flows through the adjoint kernel, so any torch optimizer trains all per-step taps
and the splitting ratio on the device.
"""
from __future__ import annotations

import math
import os
from typing import List, Optional

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


def _save_state(path: str, model, opt, it: int, scale: float, losses: List[float]) -> None:
    """Training state after `it` iterations as one .npz, written atomically (temporary file, then
    rename), so an interrupted write never leaves a half state behind."""
    arrays = {"taps": model.taps.detach().cpu().numpy(),
              "ratio": np.asarray(float(model.ratio.detach())),
              "iteration": np.asarray(it), "lr_scale": np.asarray(scale),
              "losses": np.asarray(losses, dtype=np.float64)}
    for g, param in enumerate((model.taps, model.ratio)):
        st = opt.state.get(param, {})
        if st:
            arrays[f"adam{g}_step"] = np.asarray(float(st["step"]))
            arrays[f"adam{g}_m"] = st["exp_avg"].detach().cpu().numpy()
            arrays[f"adam{g}_v"] = st["exp_avg_sq"].detach().cpu().numpy()
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def _load_state(path: str, model, opt):
    """Restore taps, ratio and the Adam moments; returns (iteration, lr scale, losses)."""
    z = np.load(path)
    with torch.no_grad():
        model.taps.copy_(torch.from_numpy(z["taps"]).to(model.taps))
        model.ratio.copy_(torch.tensor(float(z["ratio"]), dtype=torch.float64).to(model.ratio))
    for g, param in enumerate((model.taps, model.ratio)):
        if f"adam{g}_step" in z:
            opt.state[param] = {
                "step": torch.tensor(float(z[f"adam{g}_step"])),
                "exp_avg": torch.from_numpy(z[f"adam{g}_m"]).to(param),
                "exp_avg_sq": torch.from_numpy(z[f"adam{g}_v"]).to(param)}
    return int(z["iteration"]), float(z["lr_scale"]), [float(v) for v in z["losses"]]


def adam_fit(model, x_rx, loss_fn, iters: int = 200, lr_taps: float = 1e-2,
             lr_ratio: float = 1e-2, checkpoint: Optional[str] = None,
             every: int = 25) -> List[float]:
    """Adam on the taps (learning rate relative to their largest magnitude) and the ratio.

    Under torch.distributed each rank passes its own realizations (equal counts); the gradients
    are averaged over ranks in FP64 before every update, so all ranks keep identical taps and the
    update is the one of the whole data set.  The returned losses are the rank's own.

    checkpoint: path of a .npz training state (taps, ratio, Adam moments and step counts, the
    iteration, the learning-rate scale and the losses so far), written every `every`
    iterations and at the end.  If the file exists when the call starts, training resumes from
    it and runs until `iters` iterations in all, continuing exactly as an uninterrupted run
    would.  Under torch.distributed only rank 0 writes it; every rank may read it."""
    from . import distributed
    scale = float(model.taps.detach().abs().max())
    scale = distributed.max_over_ranks(scale)                 # the same learning rate everywhere
    opt = torch.optim.Adam([{"params": [model.taps], "lr": lr_taps * scale},
                            {"params": [model.ratio], "lr": lr_ratio}],
                           betas=(0.9, 0.999))
    losses: List[float] = []
    start = 0
    if checkpoint is not None and os.path.exists(checkpoint):
        start, scale, losses = _load_state(checkpoint, model, opt)
        opt.param_groups[0]["lr"] = lr_taps * scale           # the original run's scale
    writer = distributed.rank() == 0
    for it in range(start, iters):
        opt.zero_grad(set_to_none=True)
        loss = loss_fn(model(x_rx))
        loss.backward()
        distributed.average_gradients_([model.taps, model.ratio])
        opt.step()
        losses.append(float(loss.detach()))
        done = it + 1
        if checkpoint is not None and writer and (done % max(1, every) == 0 or done == iters):
            _save_state(checkpoint, model, opt, done, scale, losses)
    return losses


def snr_db_from_mse(mse: float) -> float:
    return -10.0 * math.log10(mse)
