"""The device status path (cbessfm_set_wait_limit, cbessfm_get_status): a staging wait that runs
out sets the plan's status bit and the kernel returns with its context intact.

The wait bound is shortened, never removed: with a bound of 0 each wait is one non-blocking test
of the block's mbarrier right after its bulk copy was issued, which cannot have landed yet, so
the wait gives up; the CTA then waits (with the default bound) for its copies in flight and
returns.  Nothing faults or hangs, and the next launch with the default bound is correct."""
import pytest

from parity_utils import Case, random_field, case_taps, make_plan, to_storage

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_fft,n_sb", [(256, 3), (1024, 5)])
def test_wait_limit_runs_out_and_reports_timeout(n_fft, n_sb):
    import torch
    from paper_2409_14489_gb300 import cbessfm
    case = Case(n_sb, n_fft, n_fft // 4, 2, 5, 0.3, 3 * n_sb * n_fft + 17, batch=2,
                sample_rate=64e9 * n_sb, seed=11)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    want = plan.backpropagate(x)
    assert plan.status() == cbessfm.OK
    plan.set_wait_limit(0)
    y = torch.zeros_like(x)
    plan.backpropagate(x, y)
    assert plan.status() == cbessfm.ERR_TIMEOUT
    # the status word is cleared by the read, and the default bound restores correct launches
    assert plan.status() == cbessfm.OK
    plan.set_wait_limit(-1)
    again = plan.backpropagate(x)
    assert plan.status() == cbessfm.OK
    assert torch.equal(again, want)

