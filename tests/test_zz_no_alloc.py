"""The no-allocation batched entry point (cbessfm_batch_run_noalloc), called through the C-ABI.

It serves callers that cannot allocate device memory while they run (real-time receiver threads,
memory-capped processes, plugin hosts); its work list lives in a static device array shared by
all calls.  It must give the same output as the existing entry point (cbessfm_backpropagate, one
launch per job) on two calls in a row, the second with new data, so no state of the first call
leaks into the second.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from parity_utils import Case, case_taps, random_field, make_plan, rel_l2, to_storage, from_storage

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _entry():
    from paper_2409_14489_gb300 import cbessfm
    lib = cbessfm.lib()
    fn = lib.cbessfm_batch_run_noalloc
    fn.argtypes = [ctypes.POINTER(cbessfm.JobStruct), ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return cbessfm, lib, fn


CASE_SETS = {
    # N' = 256, 3 bands, mixed lengths, steps and tap counts
    "np256": [Case(3, 256, 16, 2, 5, 0.3, 5000, sample_rate=192e9, seed=1),
              Case(3, 256, 16, 2, 5, 0.3, 777, sample_rate=192e9, seed=2),
              Case(3, 256, 16, 8, 7, 0.12, 20000, sample_rate=192e9, seed=3),
              Case(3, 256, 16, 1, 5, 0.5, 96, sample_rate=192e9, seed=4)],
    # N' = 1024, 5 bands (the two-pass layout, staged 11-tap filters next to unstaged 7-tap
    # ones), step counts in ascending order, so the call's longest-first reordering of the jobs
    # must still write each output to its own job
    "np1024": [Case(5, 1024, 256, 1, 11, 0.3, 9000, sample_rate=640e9, seed=5),
               Case(5, 1024, 256, 3, 7, 0.3, 4000, sample_rate=640e9, seed=6),
               Case(5, 1024, 256, 8, 11, 0.12, 12000, sample_rate=640e9, seed=7)],
}


@pytest.mark.parametrize("name", sorted(CASE_SETS))
def test_noalloc_batch_matches_plain_entry_point_on_two_calls(name):
    import torch
    cbessfm, lib, fn = _entry()
    cases = CASE_SETS[name]
    plans = [make_plan(c, case_taps(c)) for c in cases]
    xs = [to_storage(random_field(c)[0], 0) for c in cases]
    ys = [torch.empty_like(x) for x in xs]
    arr = (cbessfm.JobStruct * len(cases))()
    for k in range(len(cases)):
        arr[k] = cbessfm.JobStruct(plans[k].handle.value, xs[k].data_ptr(), ys[k].data_ptr(),
                                   cases[k].L)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        if call == 1:
            for x in xs:
                x.mul_(1.7)                       # different data for the second call
        for y in ys:
            y.fill_(float("nan"))
        st = fn(arr, len(cases), stream)
        assert st == 0, lib.cbessfm_last_error().decode()
        torch.cuda.synchronize()
        for k, (plan, x, y) in enumerate(zip(plans, xs, ys)):
            ref = plan.backpropagate(x)
            torch.cuda.synchronize()
            err = rel_l2(from_storage(y, 0), from_storage(ref, 0), f"noalloc/call{call}/job{k}")
            assert err <= TOL, (call, k, err)


def test_noalloc_rejects_work_beyond_its_static_limits():
    import torch
    cbessfm, lib, fn = _entry()
    c = Case(1, 64, 16, 1, 3, 0.5, 100)
    plan = make_plan(c, case_taps(c))
    x = to_storage(random_field(c)[0], 0)
    y = torch.empty_like(x)
    arr = (cbessfm.JobStruct * 65)()
    for k in range(65):
        arr[k] = cbessfm.JobStruct(plan.handle.value, x.data_ptr(), y.data_ptr(), c.L)
    assert fn(arr, 65, 0) == cbessfm.ERR_UNSUPPORTED
    assert "64" in lib.cbessfm_last_error().decode()
    c2 = Case(2, 64, 16, 1, 3, 0.5, 100, sample_rate=128e9)
    plan2 = make_plan(c2, case_taps(c2))
    arr2 = (cbessfm.JobStruct * 2)()
    arr2[0] = cbessfm.JobStruct(plan.handle.value, x.data_ptr(), y.data_ptr(), c.L)
    arr2[1] = cbessfm.JobStruct(plan2.handle.value, x.data_ptr(), y.data_ptr(), c.L)
    assert fn(arr2, 2, 0) == cbessfm.ERR_UNSUPPORTED
    assert "share" in lib.cbessfm_last_error().decode()
