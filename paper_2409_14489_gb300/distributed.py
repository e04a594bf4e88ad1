"""Multi-GPU helpers (one process per GPU, launched by torchrun).

The forward chain shards with no data-path collective: overlap-and-save blocks and realizations
are independent, so each rank backpropagates its own share and nothing crosses ranks but the
step timing.  Data-parallel coefficient training adds one reduction per iteration: the tap and
ratio gradients, averaged in FP64 so every rank applies the same update.  These helpers work with
the NCCL backend (CUDA tensors) and with gloo (CPU tensors), which the CPU tests use.
"""
from __future__ import annotations

from typing import Iterable

import torch


def is_distributed() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def rank() -> int:
    """This process's rank (0 without a process group)."""
    import torch.distributed as dist
    return dist.get_rank() if dist.is_available() and dist.is_initialized() else 0


def _device():
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous share of ``n_units`` for ``rank``: sizes differ by at most one, in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float) -> float:
    """The largest ``value`` over all ranks (the value itself without a process group)."""
    if not is_distributed():
        return float(value)
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def average_gradients_(params: Iterable[torch.nn.Parameter]) -> None:
    """Replace each parameter's gradient by its mean over ranks, summed in FP64."""
    if not is_distributed():
        return
    import torch.distributed as dist
    world = dist.get_world_size()
    dev = _device()
    for p in params:
        if p.grad is None:
            continue
        g = p.grad.detach().to(device=dev, dtype=torch.float64)
        dist.all_reduce(g, op=dist.ReduceOp.SUM)
        p.grad.copy_((g / world).to(device=p.grad.device, dtype=p.grad.dtype))
