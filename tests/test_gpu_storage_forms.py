"""16-bit storage (FP16 / BF16, FP32 arithmetic) in the streamed form and in the differentiation
form.  Their inner fields stay complex64 (the streamed form's fields between passes, the
checkpoints): the 16-bit input is widened into the workspace and the last complex64 result is
narrowed into the output.  So a 16-bit plan must give exactly the complex64 plan's result on the
widened input, narrowed with round-to-nearest, and stay within the 16-bit tolerance of the FP64
oracle fed the same storage-rounded input."""
import math

import numpy as np
import pytest

from oracle import adjoint as oadj, dbp as odbp

from parity_utils import (Case, random_field, case_taps, oracle_params, make_plan, rel_l2,
                          to_storage, from_storage, quantize, assert_parity)

pytestmark = pytest.mark.gpu

STORAGE_TOL = {1: 3e-3, 2: 3e-3}
GTOL = 1e-4


def _plans(case, taps):
    import dataclasses
    return make_plan(case, taps), make_plan(dataclasses.replace(case, storage=0), taps)


@pytest.mark.parametrize("storage", [1, 2], ids=["fp16", "bf16"])
@pytest.mark.parametrize("case", [Case(3, 128, 32, 4, 7, 0.12, 3 * 288 + 51, sample_rate=192e9, seed=3),
                                  Case(5, 1024, 256, 3, 11, 0.3, 2 * 3840 + 77, batch=2,
                                       sample_rate=640e9, seed=5)],
                         ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_st{c.n_st}")
def test_streamed_16bit(case, storage):
    import dataclasses
    import torch
    case = dataclasses.replace(case, storage=storage)
    taps = case_taps(case)
    field = random_field(case)
    p16, p64 = _plans(case, taps)
    x16 = to_storage(field, storage)
    y16 = p16.backpropagate_streamed(x16)
    q_in = quantize(field, storage)                       # the input the 16-bit plan sees
    y64 = p64.backpropagate_streamed(to_storage(q_in, 0))
    torch.cuda.synchronize()
    assert p16.status() == 0
    # the same complex64 passes on the widened input, then one round-to-nearest narrowing
    assert torch.equal(y16, to_storage(from_storage(y64, 0), storage))
    got = from_storage(y16, storage)
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    for b in range(case.batch):
        want = odbp.dbp_mode_s(q_in[b], p, case.n_fft, case.overlap)
        assert_parity(got[b], want, STORAGE_TOL[storage], f"streamed-storage{storage}/{case}/b{b}")


@pytest.mark.parametrize("storage", [1, 2], ids=["fp16", "bf16"])
def test_gradient_16bit(storage):
    """Checkpointed forward + adjoint of a 16-bit plan: the output is the complex64 plan's,
    narrowed; grad_out and grad_in stay complex64 and the gradients match the FP64 oracle's adjoint
    at the storage-rounded input within the gradient bound."""
    import torch
    case = Case(3, 128, 32, 3, 7, 0.3, 2 * 288 + 50, batch=2, sample_rate=192e9, seed=13,
                storage=storage)
    taps = case_taps(case).astype(np.float32).astype(np.float64)
    field = random_field(case)
    p16, p64 = _plans(case, taps)
    x16 = to_storage(field, storage)
    q_in = quantize(field, storage)
    ws16 = p16.new_workspace(case.L, case.batch)
    ws64 = p64.new_workspace(case.L, case.batch)
    y16 = p16.backpropagate_checkpointed(x16, ws16)
    y64 = p64.backpropagate_checkpointed(to_storage(q_in, 0), ws64)
    torch.cuda.synchronize()
    assert torch.equal(y16, to_storage(from_storage(y64, 0), storage))
    rng = np.random.default_rng(31)
    target = (rng.standard_normal(field.shape) + 1j * rng.standard_normal(field.shape)) / math.sqrt(2)
    G = 2.0 * (from_storage(y64, 0) - target)
    gc, gr, gi = p16.grad(to_storage(G, 0), ws16)
    torch.cuda.synchronize()
    assert gi.dtype == torch.complex64
    p = oracle_params(case, taps)
    o_in = np.zeros_like(q_in)
    o_taps, o_ratio = np.zeros_like(taps), 0.0
    for b in range(case.batch):
        a, t, r = oadj.dbp_mode_b_vjp(q_in[b], p, case.n_fft, case.overlap, G[b])
        o_in[b], o_taps, o_ratio = a, o_taps + t, o_ratio + r
    assert rel_l2(gc.cpu().numpy(), o_taps, f"grad-storage{storage}/taps") <= GTOL
    assert float(gr.cpu()) == pytest.approx(o_ratio, rel=GTOL, abs=1e-3 * GTOL * np.linalg.norm(o_taps))
    assert rel_l2(from_storage(gi, 0), o_in, f"grad-storage{storage}/input") <= GTOL
