"""Per-polarization NLPR (cbessfm_set_nlpr_mode(plan, 1); Eqs. (NLPR_polx), (NLPR_poly)) on the
GPU against the oracle's per-polarization chain, mode B: rel-L2 <= 1e-5 like the Manakov form.
Switching back restores the Manakov result bit for bit.  Its gradients are in
test_gpu_adjoint_perpol.py."""
import dataclasses

import numpy as np
import pytest

from oracle import dbp as odbp
from synth import configs, signals

from parity_utils import Case, random_field, case_taps, oracle_params, make_plan, rel_l2, run_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    Case(2, 64, 16, 2, 5, 0.3, 3 * 96 + 31, sample_rate=128e9, seed=2),
    Case(3, 64, 16, 3, 7, 0.12, 4 * 144 + 13, sample_rate=192e9, seed=3),
    Case(1, 256, 64, 2, 5, 0.5, 3000, seed=5),
    Case(5, 256, 64, 2, 11, 0.3, 2 * 960 + 17, sample_rate=320e9),
    Case(5, 1024, 256, 3, 11, 0.3, 2 * 3840 + 1001, sample_rate=640e9),
    Case(2, 2048, 512, 2, 11, 0.3, 4096 + 4000, sample_rate=256e9, seed=4),
]


def _oracle_per_pol(case, taps):
    return dataclasses.replace(oracle_params(case, taps), per_pol=True)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_st{c.n_st}")
def test_per_pol_matches_oracle(case):
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    manakov = run_gpu(plan, field)
    plan.set_nlpr_mode(True)
    got = run_gpu(plan, field)
    assert plan.status() == 0
    p = _oracle_per_pol(case, taps.astype(np.float32).astype(np.float64))
    want = odbp.dbp_mode_b(field[0].astype(np.complex64).astype(np.complex128), p, case.n_fft,
                           case.overlap)
    assert rel_l2(got[0], want, f"perpol/{case}") <= TOL
    if case.n_sb > 1:
        assert not np.array_equal(got, manakov)
    else:
        assert np.array_equal(got, manakov)     # no XPM: both forms are the same arithmetic
    plan.set_nlpr_mode(False)
    assert np.array_equal(run_gpu(plan, field), manakov)


def test_per_pol_c2_size_sampled_blocks():
    wl = configs.get_workload("c2_wdm15")
    d, lk = wl.dbp, wl.link
    fields = np.stack([signals.tx_waveform(wl, p, seed=wl.seed * 1000 + k)[0]
                       for k, p in enumerate(wl.launch_dbm[-2:])])
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    taps = signals.random_taps(wl.seed, d.n_st, d.n_sb, d.ntaps, w0, spread=0.2)
    case = Case(d.n_sb, d.n_fft, d.overlap, d.n_st, d.ntaps, d.ratio, wl.signal.n_samples,
                batch=len(fields), span_length=lk.span_length, n_spans=lk.n_spans,
                sample_rate=wl.signal.sample_rate)
    plan = make_plan(case, taps)
    plan.set_nlpr_mode(True)
    f32 = fields.astype(np.complex64)
    got = run_gpu(plan, f32)
    p = _oracle_per_pol(case, taps.astype(np.float32).astype(np.float64))
    n_blocks = plan.n_blocks(case.L)
    for b in range(case.batch):
        blocks = [0, n_blocks // 2, n_blocks - 1]
        want = odbp.dbp_mode_b(f32[b].astype(np.complex128), p, d.n_fft, d.overlap, blocks=blocks)
        sel = ~np.isnan(want[:, 0])
        assert rel_l2(got[b][sel], want[sel], f"perpol/c2/realization{b}") <= TOL


def test_per_pol_in_a_batch():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    cases = [Case(3, 256, 16, 2, 5, 0.3, 5000, sample_rate=192e9, seed=3),
             Case(3, 256, 16, 4, 5, 0.3, 3000, sample_rate=192e9, seed=4)]
    jobs = []
    for k, c in enumerate(cases):
        plan = make_plan(c, case_taps(c))
        plan.set_nlpr_mode(k == 0)
        x = torch.from_numpy(random_field(c)[0].astype(np.complex64)).cuda()
        jobs.append((plan, x, torch.empty_like(x)))
    batch = cbessfm.Batch(jobs)
    batch.run()
    torch.cuda.synchronize()
    for plan, x, y in jobs:
        assert torch.equal(y, plan.backpropagate(x))
