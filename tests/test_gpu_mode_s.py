"""Streamed form (cbessfm_backpropagate_streamed: one overlap-and-save pass per step) against the
oracle's mode S: rel-L2 <= 1e-5 like the plain form.  With one step it is the plain launch bit
for bit; on a long link with a short overlap it stays close to the whole-sequence chain where
the plain form (whole chain per block) does not."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import dbp as odbp
from synth import signals

from parity_utils import (Case, random_field, case_taps, oracle_params, make_plan, rel_l2,
                          to_storage, from_storage)

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    Case(1, 64, 16, 2, 5, 0.5, 4 * 48 + 6, seed=1),
    Case(2, 64, 16, 3, 5, 0.3, 3 * 96 + 32, sample_rate=128e9, seed=2),
    Case(3, 128, 32, 4, 7, 0.12, 3 * 288 + 51, sample_rate=192e9, seed=3),
    Case(5, 256, 64, 3, 11, 0.3, 2 * 960 + 20, sample_rate=320e9, seed=4),
    Case(5, 1024, 256, 2, 11, 0.3, 2 * 3840 + 1000, sample_rate=640e9, seed=5),
    Case(2, 2048, 512, 3, 11, 0.3, 2 * 3072 + 78, batch=2, sample_rate=256e9, seed=6),
]


def _run_streamed(plan, field):
    import torch
    x = to_storage(field, 0)
    y = plan.backpropagate_streamed(x)
    torch.cuda.synchronize()
    return from_storage(y, 0)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_st{c.n_st}_b{c.batch}")
def test_streamed_matches_oracle_mode_s(case):
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    got = _run_streamed(plan, field)
    assert plan.status() == 0
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    for b in range(case.batch):
        want = odbp.dbp_mode_s(field[b].astype(np.complex64).astype(np.complex128), p,
                               case.n_fft, case.overlap)
        assert rel_l2(got[b], want, f"streamed/{case}/b{b}") <= TOL


def test_streamed_single_step_is_the_plain_launch():
    import torch
    case = Case(3, 256, 64, 1, 7, 0.3, 5000, sample_rate=192e9, seed=7)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    assert torch.equal(plan.backpropagate_streamed(x), plan.backpropagate(x))


def test_streamed_per_polarization_matches_oracle():
    case = Case(3, 128, 32, 3, 7, 0.3, 3 * 288 + 51, sample_rate=192e9, seed=8)
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    plan.set_nlpr_mode(True)
    got = _run_streamed(plan, field)
    p = dataclasses.replace(oracle_params(case, taps.astype(np.float32).astype(np.float64)),
                            per_pol=True)
    want = odbp.dbp_mode_s(field[0].astype(np.complex64).astype(np.complex128), p, case.n_fft,
                           case.overlap)
    assert rel_l2(got[0], want, "streamed/per-pol") <= TOL


def test_streamed_needs_only_one_steps_memory():
    """8 x 80 km at 96 GS/s, 3 subbands, N' = 256, N'_ov = 64: each pass's overlap covers one
    step, the plain form's does not cover the link."""
    n_sb, n_fft, overlap, n_st = 3, 256, 64, 8
    rate, L = 96e9, 3 * 2048
    rng = np.random.default_rng(11)
    X = np.fft.fft(0.05 * (rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2))), axis=0)
    X[np.abs(np.fft.fftfreq(L) * rate) > 0.4 * rate] = 0
    field = np.fft.ifft(X, axis=0)
    taps = signals.random_taps(5, n_st, n_sb, 5, 0.5, spread=0.3)
    case = Case(n_sb, n_fft, overlap, n_st, 5, 0.3, L, span_length=80e3, n_spans=n_st,
                sample_rate=rate)
    plan = make_plan(case, taps)
    import torch
    x = to_storage(field[None], 0)
    ys = from_storage(plan.backpropagate_streamed(x), 0)[0]
    yb = from_storage(plan.backpropagate(x), 0)[0]
    torch.cuda.synchronize()
    ref = odbp.dbp_mode_u(field.astype(np.complex64).astype(np.complex128),
                          oracle_params(case, taps.astype(np.float32).astype(np.float64)))
    e_s, e_b = rel_l2(ys, ref), rel_l2(yb, ref)
    assert e_s < 0.1 * e_b and e_s < 1e-2, (e_s, e_b)


def test_streamed_argument_checks():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    case = Case(2, 64, 16, 3, 5, 0.3, 500, sample_rate=128e9)
    plan = make_plan(case, case_taps(case))
    x = to_storage(random_field(case), 0)
    ws = torch.empty(plan.streamed_workspace_size(case.L, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(cbessfm.CBESSFMError, match="overlaps"):
        plan.backpropagate_streamed(x, out=x, workspace=ws)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(cbessfm.CBESSFMError, match="workspace"):
        plan.backpropagate_streamed(x, workspace=small)
