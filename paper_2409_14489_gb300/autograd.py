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
    """y = DBP(x; taps, ratio).  Each call checkpoints into a workspace of its own, which the
    autograd graph keeps until the call's backward, so several calls may precede their backward
    passes (a loss summed over two batches).  The backward pass reloads the call's taps and
    ratio into the plan if a later call changed them, and an in-place change of the taps between
    a call and its backward raises, as for any tensor that autograd saves."""

    @staticmethod
    def forward(ctx, x, taps, ratio, module):
        ratio_value = float(ratio.detach())
        token = module._load_plan(taps, ratio_value)
        batch, L = cbessfm.Plan._shape(x)
        ws = module.plan.new_workspace(L, batch)
        y = module.plan.backpropagate_checkpointed(x.contiguous(), ws)
        ctx.save_for_backward(taps)
        ctx.module, ctx.ws, ctx.token, ctx.ratio_value = module, ws, token, ratio_value
        ctx.taps_dtype = taps.dtype
        ctx.ratio_dtype = ratio.dtype
        return y

    @staticmethod
    def backward(ctx, gy):
        (taps,) = ctx.saved_tensors
        module = ctx.module
        module._reload_plan(ctx.token, taps, ctx.ratio_value)
        gc, gr, gi = module.plan.grad(gy.contiguous(), ctx.ws, want_input=ctx.needs_input_grad[0],
                                      want_ratio=ctx.needs_input_grad[2])
        return (gi, gc.to(ctx.taps_dtype), gr.to(ctx.ratio_dtype) if gr is not None else None,
                None)


class CBESSFM(torch.nn.Module):
    """CB-ESSFM DBP with trainable per-step taps and splitting ratio (complex64 fields).

    ``plan`` wraps an existing plan instead of creating one from the other arguments (the plan
    must match them); ``device`` holds the parameters."""

    def __init__(self, link, bands: int, steps: int, ratio: float, taps, n_fft: int,
                 overlap: int, *, plan=None, device="cuda"):
        super().__init__()
        taps = torch.as_tensor(np.asarray(taps), dtype=torch.float32)
        self.plan = plan if plan is not None else cbessfm.Plan(link, bands, steps, ratio,
                                                                taps.numpy(), n_fft, overlap)
        self.taps = torch.nn.Parameter(taps.to(device))
        self.ratio = torch.nn.Parameter(torch.tensor(float(ratio), dtype=torch.float64,
                                                     device=device))
        self._token = 0       # counts the taps/ratio states loaded into the plan
        self._loaded = 0      # the state the plan holds now

    def _load_plan(self, taps, ratio: float) -> int:
        """Loads taps and ratio into the plan; returns the token naming this state."""
        self.plan.set_coeffs(taps.detach().to(torch.float32).contiguous())
        self.plan.set_ratio(ratio)
        self._token += 1
        self._loaded = self._token
        return self._token

    def _reload_plan(self, token: int, taps, ratio: float) -> None:
        if self._loaded != token:
            self.plan.set_coeffs(taps.detach().to(torch.float32).contiguous())
            self.plan.set_ratio(ratio)
            self._loaded = token

    def forward(self, x):
        if not 0.0 <= float(self.ratio.detach()) <= 1.0:
            with torch.no_grad():
                self.ratio.clamp_(0.0, 1.0)
        if torch.is_grad_enabled() and (x.requires_grad or self.taps.requires_grad
                                        or self.ratio.requires_grad):
            return CBESSFMFunction.apply(x, self.taps, self.ratio, self)
        # nothing to differentiate: the plain forward, without checkpoints
        self._load_plan(self.taps, float(self.ratio.detach()))
        return self.plan.backpropagate(x.contiguous())
