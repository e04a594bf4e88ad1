"""PyTorch autograd integration of the differentiation form.

``CBESSFMFunction`` runs the checkpointed forward kernel and, in backward, the adjoint kernel
(gradients of every step's taps, of the splitting ratio and of the input field; taps and ratio
gradients summed over blocks in FP64).  ``CBESSFM`` is an ``nn.Module`` holding the taps and the
ratio as parameters, so the paper's offline coefficient optimization (Sec. III-B) becomes plain
gradient descent on the device (e.g. ``torch.optim.Adam``).

All arithmetic runs in the library's kernels; PyTorch supplies memory, streams and the optimizer.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cbessfm


class CBESSFMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, taps, ratio, module):
        plan = module.plan
        plan.set_coeffs(taps.detach().to(torch.float32).contiguous())
        plan.set_ratio(float(ratio.detach()))
        batch, L = cbessfm.Plan._shape(x)
        ws = module.workspace(L, batch)
        y = plan.backpropagate_checkpointed(x.contiguous(), ws)
        ctx.module = module
        ctx.taps_dtype = taps.dtype
        ctx.ratio_dtype = ratio.dtype
        return y

    @staticmethod
    def backward(ctx, gy):
        module = ctx.module
        batch, L = cbessfm.Plan._shape(gy)
        ws = module.workspace(L, batch)
        gc, gr, gi = module.plan.grad(gy.contiguous(), ws, want_input=ctx.needs_input_grad[0],
                                      want_ratio=ctx.needs_input_grad[2])
        return (gi, gc.to(ctx.taps_dtype), gr.to(ctx.ratio_dtype) if gr is not None else None,
                None)


class CBESSFM(torch.nn.Module):
    """CB-ESSFM DBP with trainable per-step taps and splitting ratio (complex64 fields)."""

    def __init__(self, link, bands: int, steps: int, ratio: float, taps, n_fft: int,
                 overlap: int):
        super().__init__()
        taps = torch.as_tensor(np.asarray(taps), dtype=torch.float32)
        self.plan = cbessfm.Plan(link, bands, steps, ratio, taps.numpy(), n_fft, overlap)
        self.taps = torch.nn.Parameter(taps.cuda())
        self.ratio = torch.nn.Parameter(torch.tensor(float(ratio), dtype=torch.float64,
                                                     device="cuda"))
        self._ws = None

    def workspace(self, n_samples: int, batch: int):
        need = self.plan.workspace_size(n_samples, batch)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        return self._ws

    def forward(self, x):
        with torch.no_grad():
            self.ratio.clamp_(0.0, 1.0)
        return CBESSFMFunction.apply(x, self.taps, self.ratio, self)
