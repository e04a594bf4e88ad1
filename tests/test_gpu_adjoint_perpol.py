"""Differentiation form of the per-polarization NLPR (Eqs. (NLPR_polx), (NLPR_poly)): the adjoint
kernel after a checkpointed per-polarization forward, against the FP64 oracle's adjoint of the same
chain (oracle.adjoint with per_pol) and against central finite differences of the FP64 oracle.
Tolerance: 1e-4 relative, the bound the Manakov form's gradients meet."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import adjoint as oadj, dbp as odbp

from parity_utils import Case, random_field, case_taps, oracle_params, make_plan, rel_l2, \
    to_storage, from_storage

pytestmark = pytest.mark.gpu

GTOL = 1e-4

CASES = [
    Case(2, 64, 16, 2, 5, 0.3, 3 * 96 + 31, sample_rate=128e9, seed=2),
    Case(3, 128, 32, 3, 7, 0.12, 2 * 288 + 50, sample_rate=192e9, seed=3),
    Case(5, 256, 64, 2, 11, 0.3, 2 * 960 + 17, sample_rate=320e9, seed=4),
    Case(2, 512, 128, 3, 9, 0.7, 2 * 768 + 99, batch=2, sample_rate=128e9, seed=6),
]


def _per_pol_params(case, taps):
    return dataclasses.replace(oracle_params(case, taps), per_pol=True)


def _gpu_grad(case, taps, field, target, want_ratio=True):
    import torch
    plan = make_plan(case, taps)
    plan.set_nlpr_mode(True)
    ws = plan.new_workspace(case.L, case.batch)
    y = plan.backpropagate_checkpointed(to_storage(field, 0), ws)
    torch.cuda.synchronize()
    y_np = from_storage(y, 0)
    G = 2.0 * (y_np - target)                                  # d/d(out) of sum |out - t|^2
    gc, gr, gi = plan.grad(to_storage(G, 0), ws, want_ratio=want_ratio)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return y_np, G, gc.cpu().numpy(), (float(gr.cpu()) if gr is not None else None), \
        from_storage(gi, 0)


def _target(case, field):
    rng = np.random.default_rng(case.seed + 100)
    return (rng.standard_normal(field.shape) + 1j * rng.standard_normal(field.shape)) / math.sqrt(2)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_st{c.n_st}_b{c.batch}")
def test_per_pol_adjoint_matches_oracle_adjoint(case):
    taps = case_taps(case).astype(np.float32).astype(np.float64)
    field = random_field(case).astype(np.complex64).astype(np.complex128)
    target = _target(case, field)
    y, G, gc, gr, gi = _gpu_grad(case, taps, field, target)
    p = _per_pol_params(case, taps)
    # the checkpointed forward is the per-polarization chain itself
    for b in range(case.batch):
        ref = odbp.dbp_mode_b(field[b], p, case.n_fft, case.overlap)
        assert rel_l2(y[b], ref, f"perpol-ckpt-forward/{case}") <= 1e-5
    o_in = np.zeros_like(field)
    o_taps, o_ratio = np.zeros_like(taps), 0.0
    for b in range(case.batch):
        a, t, r = oadj.dbp_mode_b_vjp(field[b], p, case.n_fft, case.overlap, G[b])
        o_in[b], o_taps, o_ratio = a, o_taps + t, o_ratio + r
    assert rel_l2(gc, o_taps, f"perpol-adjoint/taps/{case}") <= GTOL
    assert abs(gr - o_ratio) <= GTOL * max(abs(o_ratio), 1e-3 * np.linalg.norm(o_taps)), (gr, o_ratio)
    rel_l2(np.array([gr]), np.array([o_ratio]), f"perpol-adjoint/ratio/{case}")
    assert rel_l2(gi, o_in, f"perpol-adjoint/input/{case}") <= GTOL


def test_per_pol_adjoint_differs_from_manakov_where_the_coupling_taps_act():
    """The per-polarization gradient is not the Manakov one: with coupling taps and unequal x and
    y powers the two oracle adjoints differ by far more than the tolerance, and the GPU follows
    the per-polarization one (a kernel that ignored the mode would fail here)."""
    case = CASES[1]
    taps = case_taps(case).astype(np.float32).astype(np.float64)
    field = random_field(case).astype(np.complex64).astype(np.complex128)
    field[..., 1] *= 0.3                                       # unequal polarization powers
    target = _target(case, field)
    _, G, gc, _, _ = _gpu_grad(case, taps, field, target, want_ratio=False)
    _, t_pp, _ = oadj.dbp_mode_b_vjp(field[0], _per_pol_params(case, taps), case.n_fft,
                                     case.overlap, G[0])
    _, t_mk, _ = oadj.dbp_mode_b_vjp(field[0], oracle_params(case, taps), case.n_fft,
                                     case.overlap, G[0])
    assert rel_l2(t_mk, t_pp) > 100 * GTOL
    assert rel_l2(gc, t_pp, "perpol-adjoint/taps-only") <= GTOL


def test_per_pol_adjoint_matches_finite_differences_of_oracle():
    case = Case(3, 64, 16, 2, 5, 0.3, 3 * 144 + 13, sample_rate=192e9, seed=9)
    taps = case_taps(case).astype(np.float32).astype(np.float64)
    field = random_field(case).astype(np.complex64).astype(np.complex128)
    field[..., 1] *= 0.5
    target = _target(case, field)
    _, _, gc, gr, _ = _gpu_grad(case, taps, field, target)

    def loss(tp, rho):
        p = odbp.ChainParams(case.beta2, case.sample_rate, case.link_length, case.n_sb, rho, tp,
                             per_pol=True)
        out = odbp.dbp_mode_b(field[0], p, case.n_fft, case.overlap)
        return float(np.sum(np.abs(out - target[0]) ** 2))

    h = 1e-4
    for ix in [(0, 0, 0, 2), (1, 1, 2, 0), (0, 2, 1, 4), (1, 0, 2, 2)]:
        tp, tm = taps.copy(), taps.copy()
        tp[ix] += h
        tm[ix] -= h
        fd = (loss(tp, case.ratio) - loss(tm, case.ratio)) / (2 * h)
        assert gc[ix] == pytest.approx(fd, rel=GTOL, abs=GTOL * np.max(np.abs(gc))), ix
    fd = (loss(taps, case.ratio + h) - loss(taps, case.ratio - h)) / (2 * h)
    assert gr == pytest.approx(fd, rel=GTOL, abs=1e-6 * np.max(np.abs(gc)))


def test_per_pol_gradient_refused_where_its_rows_do_not_fit():
    """Five subbands of N' = 1024: the per-polarization adjoint's extra rows exceed shared memory,
    so the checkpointed forward refuses the plan with CBESSFM_ERR_UNSUPPORTED (the Manakov form of
    the same plan is tested on the differentiation workload)."""
    import torch
    from paper_2409_14489_gb300 import cbessfm
    case = Case(5, 1024, 256, 2, 11, 0.3, 2 * 3840 + 1001, sample_rate=640e9, seed=7)
    plan = make_plan(case, case_taps(case))
    plan.set_nlpr_mode(True)
    x = torch.from_numpy(random_field(case)[0].astype(np.complex64)).cuda()
    ws = plan.new_workspace(case.L, 1)
    with pytest.raises(cbessfm.CBESSFMError, match="per-polarization") as err:
        plan.backpropagate_checkpointed(x, ws)
    assert err.value.status == cbessfm.ERR_UNSUPPORTED
