"""Multi-rank host logic on CPU with the gloo backend (world size 2): work sharding, the timing
reduction of the benchmark, and data-parallel coefficient training (gradients averaged in FP64
over ranks give every rank the same taps, equal to training on all the data in one process).
The GPU kernels are not involved; the model here is a small differentiable stand-in."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2409_14489_gb300 import distributed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class _StandIn(torch.nn.Module):
    """taps and ratio parameters like CBESSFM; y = x * (taps . basis) + ratio * x^2."""

    def __init__(self):
        super().__init__()
        self.taps = torch.nn.Parameter(torch.tensor([[0.3, -0.2, 0.1]], dtype=torch.float32))
        self.ratio = torch.nn.Parameter(torch.tensor(0.5, dtype=torch.float64))

    def forward(self, x):
        basis = torch.stack([x, x.roll(1, -1), x.roll(-1, -1)], dim=-1)
        return (basis * self.taps[0]).sum(-1) + self.ratio.float() * x ** 2


def _data(rank, n_per_rank):
    g = torch.Generator().manual_seed(100 + rank)
    x = torch.randn(n_per_rank, 16, generator=g)
    target = 0.7 * x + 0.05 * x.roll(1, -1) - 0.2 * x ** 2
    return x, target


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        out["shard"] = list(distributed.shard(11, rank, world))
        out["max"] = distributed.max_over_ranks(1.5 + rank)
        from paper_2409_14489_gb300 import train
        model = _StandIn()
        x, target = _data(rank, 4)
        losses = train.adam_fit(model, x, lambda y: torch.mean((y - target) ** 2), iters=30,
                                lr_taps=0.05, lr_ratio=0.02)
        out["taps"] = model.taps.detach().numpy().copy()
        out["ratio"] = float(model.ratio.detach())
        out["loss_drop"] = losses[-1] < losses[0]
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_reduce_and_train_data_parallel():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # sharding covers every unit once, in order, balanced
    assert res[0]["shard"] + res[1]["shard"] == list(range(11))
    assert abs(len(res[0]["shard"]) - len(res[1]["shard"])) <= 1
    # the benchmark's timing reduction is the maximum over ranks
    assert res[0]["max"] == res[1]["max"] == 2.5
    # identical parameters on both ranks ...
    np.testing.assert_array_equal(res[0]["taps"], res[1]["taps"])
    assert res[0]["ratio"] == res[1]["ratio"]
    assert res[0]["loss_drop"] and res[1]["loss_drop"]
    # ... equal to one process training on both ranks' data (mean loss over equal shards)
    from paper_2409_14489_gb300 import train
    model = _StandIn()
    xs, ts = zip(*(_data(r, 4) for r in range(world)))
    x, target = torch.cat(xs), torch.cat(ts)
    train.adam_fit(model, x, lambda y: torch.mean((y - target) ** 2), iters=30, lr_taps=0.05,
                   lr_ratio=0.02)
    np.testing.assert_allclose(res[0]["taps"], model.taps.detach().numpy(), rtol=1e-5, atol=1e-7)
    assert res[0]["ratio"] == pytest.approx(float(model.ratio.detach()), rel=1e-6)


def test_shard_edge_cases_and_single_process_fallbacks():
    assert list(distributed.shard(0, 0, 3)) == []
    assert [len(distributed.shard(7, r, 3)) for r in range(3)] == [3, 2, 2]
    with pytest.raises(ValueError):
        distributed.shard(5, 2, 2)
    assert distributed.max_over_ranks(3.25) == 3.25            # no process group
    p = torch.nn.Parameter(torch.ones(2))
    p.grad = torch.full((2,), 0.5)
    distributed.average_gradients_([p])
    assert torch.equal(p.grad, torch.full((2,), 0.5))


class _InjectedFailure(RuntimeError):
    pass


def _failing_worker(rank, world, port, q):
    """Rank 1's loss raises in its 4th iteration (before that iteration's gradient all-reduce);
    rank 0 must see an error from its next collective instead of waiting forever."""
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    from paper_2409_14489_gb300 import train
    model = _StandIn()
    x, target = _data(rank, 4)
    calls = [0]

    def loss_fn(y):
        calls[0] += 1
        if rank == 1 and calls[0] == 4:
            raise _InjectedFailure("injected failure on rank 1")
        return torch.mean((y - target) ** 2)

    try:
        train.adam_fit(model, x, loss_fn, iters=30, lr_taps=0.05, lr_ratio=0.02)
        q.put((rank, "finished", calls[0]))
    except Exception as e:                      # noqa: BLE001 -- reported to the test
        q.put((rank, type(e).__name__, calls[0]))
    # no destroy_process_group: a failed rank just leaves, as a crashed one would


def test_a_failed_rank_ends_the_others_collective_with_an_error():
    """Failure detection on the host: one rank of a data-parallel training run fails between
    steps; the survivor's next gradient all-reduce ends with an error (peer gone or the process
    group's 20 s timeout) rather than hanging, and it had not taken another step."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = {r: (status, n) for r, status, n in (q.get(timeout=120) for _ in range(world))}
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert res[1] == ("_InjectedFailure", 4)
    status0, calls0 = res[0]
    assert status0 != "finished", res
    assert calls0 == 4                          # its 4th step's all-reduce is where it stopped
