"""Host-resident fields (cbessfm_backpropagate_host): the pipelined copies and the launches over
ranges of OLS blocks give the device path's result bit for bit, for any launch size (ranges
that start and end inside a realization included), copy grouping and storage type."""
import pytest

from parity_utils import Case, random_field, case_taps, make_plan, to_storage

pytestmark = pytest.mark.gpu


def _pinned(x):
    import torch
    h_in = x.cpu().pin_memory()
    return h_in, torch.empty_like(h_in).pin_memory()


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("launch_blocks", [0, 1, 5, 7, 13, 54, 55, 1000])
def test_host_pipeline_equals_device_path(storage, launch_blocks):
    """5 realizations of 6000 samples, V = 576: 11 blocks each, 55 in all."""
    import torch
    case = Case(3, 256, 64, 3, 7, 0.3, 6000, batch=5, sample_rate=192e9, seed=3, storage=storage)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), storage)
    want = plan.backpropagate(x)
    h_in, h_out = _pinned(x)
    d_in, d_out = torch.empty_like(x), torch.empty_like(x)
    plan.backpropagate_host(h_in, h_out, d_in, d_out, launch_blocks=launch_blocks)
    torch.cuda.synchronize()
    assert torch.equal(h_out, want.cpu())
    assert plan.status() == 0


def test_host_pipeline_automatic_launches_span_several_waves():
    """Two c2-sized realizations (5 subbands, N' = 1024: one resident block per SM, 342 blocks):
    the automatic sizing runs a first launch of one wave and a second of up to two waves, and
    the copies out follow each realization's last block."""
    import torch
    case = Case(5, 1024, 256, 2, 11, 0.3, 655360, batch=2, sample_rate=640e9, seed=7)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    want = plan.backpropagate(x).cpu()
    h_in, h_out = _pinned(x)
    d_in, d_out = torch.empty_like(x), torch.empty_like(x)
    plan.backpropagate_host(h_in, h_out, d_in, d_out)
    torch.cuda.synchronize()
    assert torch.equal(h_out, want)
    assert plan.status() == 0


def test_host_pipeline_groups_many_realizations():
    """70 realizations (more than the 64 copy groups: two per group), 2 blocks each."""
    import torch
    case = Case(2, 128, 32, 2, 5, 0.3, 300, batch=70, sample_rate=128e9, seed=5)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    want = plan.backpropagate(x).cpu()
    h_in, h_out = _pinned(x)
    d_in, d_out = torch.empty_like(x), torch.empty_like(x)
    for lb in (0, 3, 17):
        h_out.zero_()
        plan.backpropagate_host(h_in, h_out, d_in, d_out, launch_blocks=lb)
        torch.cuda.synchronize()
        assert torch.equal(h_out, want)


def test_host_pipeline_pageable_memory_and_repeat_calls():
    import torch
    case = Case(2, 128, 32, 2, 5, 0.3, 3000, batch=3, sample_rate=128e9, seed=4)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    want = plan.backpropagate(x).cpu()
    h_in = x.cpu()                                   # pageable: still correct, less overlap
    d_in, d_out = torch.empty_like(x), torch.empty_like(x)
    for _ in range(3):
        h_out = torch.zeros_like(h_in)
        plan.backpropagate_host(h_in, h_out, d_in, d_out, launch_blocks=4)
        torch.cuda.synchronize()
        assert torch.equal(h_out, want)


def test_host_pipeline_argument_checks():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    case = Case(2, 128, 32, 2, 5, 0.3, 3000, batch=2, sample_rate=128e9, seed=6)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    h_in, h_out = _pinned(x)
    d_in = torch.empty_like(x)
    with pytest.raises(cbessfm.CBESSFMError, match="launch_blocks"):
        plan.backpropagate_host(h_in, h_out, d_in, torch.empty_like(x), launch_blocks=-1)
    with pytest.raises(cbessfm.CBESSFMError, match="overlaps"):
        plan.backpropagate_host(h_in, h_out, d_in, d_in)
