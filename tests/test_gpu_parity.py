"""Parity of the CUDA forward chain (cbessfm_backpropagate) with the FP64 oracle (mode B).

Tolerance: relative L2 error <= 1e-5 for complex64 (the bound stated for the FP32 path), on
every compared sample.  Small cases span several blocks plus a ragged tail and exercise every
supported N' and several subband counts, step counts, tap counts and splitting ratios; the
full-size workloads compare sampled blocks (the oracle computes those blocks one by one).
"""
import math

import numpy as np
import pytest

from oracle import channel, dbp as odbp, evaluate
from synth import configs, signals

from parity_utils import (Case, random_field, case_taps, oracle_params, make_plan, run_gpu, rel_l2,
                          quantize, assert_parity)

pytestmark = pytest.mark.gpu

TOL = 1e-5

SMALL_CASES = [
    # n_sb, n_fft, overlap, n_st, ntaps, ratio, L
    Case(1, 16, 4, 1, 3, 0.5, 5 * 12 + 7),
    Case(1, 32, 8, 2, 5, 0.3, 4 * 24 + 5, sample_rate=32e9),
    Case(2, 64, 16, 2, 5, 0.3, 3 * 96 + 31, sample_rate=128e9),
    Case(3, 64, 16, 3, 7, 0.12, 4 * 144 + 13, sample_rate=192e9),
    Case(5, 128, 32, 2, 11, 0.3, 3 * 480 + 99, sample_rate=320e9),
    Case(1, 256, 64, 1, 5, 0.5, 8192),
    Case(5, 256, 64, 2, 11, 0.3, 2 * 960 + 17, sample_rate=320e9),
    Case(4, 512, 128, 3, 9, 1.0, 2 * 1536 + 300, sample_rate=256e9),
    Case(5, 1024, 256, 2, 11, 0.3, 2 * 3840 + 1001, sample_rate=640e9),
    Case(2, 2048, 512, 2, 11, 0.0, 2 * 3072 + 77, sample_rate=128e9),
    Case(2, 2048, 512, 1, 11, 0.3, 4096 + 4000, sample_rate=256e9, seed=4),
    Case(5, 2048, 512, 2, 11, 0.3, 10240 + 4000, sample_rate=640e9),
    Case(3, 32, 8, 0, 1, 0.5, 200, sample_rate=96e9),             # EDC (no NLPR steps)
    Case(2, 64, 16, 4, 1, 0.5, 333, sample_rate=128e9),           # single-tap (OSSFM-like)
    Case(1, 64, 0, 2, 5, 0.5, 64 * 3),                            # no overlap
    Case(2, 64, 16, 2, 5, 0.3, 100, batch=3, sample_rate=128e9),  # L < block: multiple wraps
    Case(1, 16, 4, 3, 3, 0.5, 1),                                 # one sample
]


@pytest.mark.parametrize("case", SMALL_CASES, ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_st{c.n_st}_"
                         f"t{c.ntaps}_r{c.ratio}_L{c.L}_b{c.batch}")
def test_forward_matches_oracle_small(case):
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    got = run_gpu(plan, field)
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    for b in range(case.batch):
        want = odbp.dbp_mode_b(field[b].astype(np.complex64).astype(np.complex128), p,
                               case.n_fft, case.overlap)
        assert_parity(got[b], want, TOL, f"small/{case}/b{b}")
    assert plan.status() == 0


# Shapes at the edges of what plan_create accepts: more subbands (up to 16 at N' = 256, 10 at
# 512) and long filters (up to N'/2 taps: the windowed FIR's general chunk loop and wide halos).
# Taps scale as 1/ntaps so the nonlinear phase per step stays comparable.
WIDE_CASES = [
    Case(8, 256, 64, 2, 21, 0.3, 2 * 8 * 192 + 77, sample_rate=512e9, tap_scale=1.0 / 21),
    Case(16, 256, 64, 2, 11, 0.3, 2 * 16 * 192 + 55, sample_rate=1024e9, tap_scale=1.0 / 11),
    Case(10, 512, 128, 2, 45, 0.3, 2 * 10 * 384 + 333, sample_rate=640e9, tap_scale=1.0 / 45),
    Case(5, 1024, 256, 2, 45, 0.3, 2 * 3840 + 555, sample_rate=640e9, tap_scale=1.0 / 45),
    Case(2, 256, 64, 2, 127, 0.5, 3 * 384 + 11, sample_rate=128e9, tap_scale=1.0 / 127),
    Case(3, 1024, 256, 1, 511, 0.5, 2 * 2304 + 99, sample_rate=192e9, tap_scale=1.0 / 511),
    Case(5, 2048, 512, 1, 101, 0.3, 10240 + 4000, sample_rate=640e9, tap_scale=1.0 / 101),
]


@pytest.mark.parametrize("case", WIDE_CASES, ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_t{c.ntaps}")
def test_forward_matches_oracle_wide_shapes(case):
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    got = run_gpu(plan, field)
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    want = odbp.dbp_mode_b(field[0].astype(np.complex64).astype(np.complex128), p, case.n_fft,
                           case.overlap)
    assert_parity(got[0], want, TOL, f"wide/{case}")
    assert plan.status() == 0


LAYOUT_CASES = [
    Case(1, 16, 4, 3, 3, 0.5, 5 * 12 + 7),                       # one-pass FFT
    Case(3, 64, 16, 3, 7, 0.12, 4 * 144 + 13, sample_rate=192e9),  # two-pass FFT
    Case(1, 256, 64, 2, 5, 0.5, 3000, batch=2),                   # several blocks per CTA
    Case(5, 1024, 256, 3, 11, 0.3, 2 * 3840 + 1001, sample_rate=640e9),
    Case(2, 2048, 512, 2, 11, 0.3, 4096 + 4000, sample_rate=256e9, seed=4),
]


@pytest.mark.parametrize("case", LAYOUT_CASES, ids=lambda c: f"sb{c.n_sb}_np{c.n_fft}_st{c.n_st}")
def test_shared_memory_layouts_agree_bitwise(case, monkeypatch):
    """Every shared-memory layout of the forward chain (ping-pong exchange arrays with two or one
    intensity buffers, separate rows, rows aliased onto the exchange array) runs the same
    arithmetic, so the outputs must be identical; the default one also meets the oracle."""
    taps = case_taps(case)
    field = random_field(case)
    outs = {}
    for lay in ("pingpong2", "pingpong1", "separate", "alias", None):
        if lay is None:
            monkeypatch.delenv("CBESSFM_SMEM_LAYOUT", raising=False)
        else:
            monkeypatch.setenv("CBESSFM_SMEM_LAYOUT", lay)
        plan = make_plan(case, taps)
        outs[lay] = run_gpu(plan, field)
        assert plan.status() == 0
    for lay, got in outs.items():
        assert np.array_equal(got, outs[None]), lay
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    want = odbp.dbp_mode_b(field[0].astype(np.complex64).astype(np.complex128), p, case.n_fft,
                           case.overlap)
    assert rel_l2(outs[None][0], want, f"layouts/{case}") <= TOL


def test_c1_channel_output_parity_and_snr():
    wl = configs.get_workload("c1_tiny")
    lk, sig, d = wl.link, wl.signal, wl.dbp
    tx, syms = signals.tx_waveform(wl, 0.0, seed=wl.seed)
    rx = channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, lk.n_spans,
                           sig.sample_rate, steps_per_span=1000)
    p_w = configs.dbm_to_watt(0.0)
    # taps act on |u|^2 in W: gamma * L_eff per step (rad/W), SSFM-init plus a perturbation
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    taps = signals.random_taps(wl.seed, d.n_st, d.n_sb, d.ntaps, w0, spread=0.2)
    case = Case(d.n_sb, d.n_fft, d.overlap, d.n_st, d.ntaps, d.ratio, sig.n_samples,
                sample_rate=sig.sample_rate)
    plan = make_plan(case, taps)
    rx32 = rx.astype(np.complex64)
    got = run_gpu(plan, rx32[None])[0]
    want = odbp.dbp_mode_b(rx32.astype(np.complex128), oracle_params(
        case, taps.astype(np.float32).astype(np.float64)), d.n_fft, d.overlap)
    assert rel_l2(got, want, "c1_channel") <= TOL
    p_pol = p_w / 2
    snr_gpu = evaluate.snr_db(evaluate.receive(got, sig.sample_rate, sig.baud, sig.rolloff, 0.0,
                                               p_pol), syms[0])
    snr_ref = evaluate.snr_db(evaluate.receive(want, sig.sample_rate, sig.baud, sig.rolloff, 0.0,
                                               p_pol), syms[0])
    assert abs(snr_gpu - snr_ref) <= 0.02


def _c2_inputs(n_real):
    wl = configs.get_workload("c2_wdm15")
    fields = []
    for k, p_dbm in enumerate(wl.launch_dbm[:n_real]):
        tx, _ = signals.tx_waveform(wl, p_dbm, seed=wl.seed * 1000 + k)
        fields.append(tx)
    return wl, np.stack(fields)


def test_c2_full_size_sampled_blocks():
    """Paper-scale workload (7 x 655,360 samples, 5 subbands, 15 steps): all realizations on the
    GPU in the benchmark's launch configuration; the oracle recomputes sampled blocks, including
    the first and last (wrapping) blocks of every realization."""
    wl, fields = _c2_inputs(7)
    d, lk = wl.dbp, wl.link
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)   # rad/W per 80 km step
    taps = signals.random_taps(wl.seed, d.n_st, d.n_sb, d.ntaps, w0, spread=0.2)
    case = Case(d.n_sb, d.n_fft, d.overlap, d.n_st, d.ntaps, d.ratio, wl.signal.n_samples,
                batch=len(fields), span_length=lk.span_length, n_spans=lk.n_spans,
                sample_rate=wl.signal.sample_rate)
    plan = make_plan(case, taps)
    f32 = fields.astype(np.complex64)
    got = run_gpu(plan, f32)
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    n_blocks = plan.n_blocks(case.L)
    rng = np.random.default_rng(7)
    for b in range(case.batch):
        blocks = sorted({0, n_blocks - 1, int(rng.integers(1, n_blocks - 1))})
        want = odbp.dbp_mode_b(f32[b].astype(np.complex128), p, d.n_fft, d.overlap, blocks=blocks)
        sel = ~np.isnan(want[:, 0])
        assert_parity(got[b][sel], want[sel], TOL, f"c2_full/realization{b}")
    assert np.isfinite(got).all()


def test_batch_entries_are_independent():
    case = Case(3, 64, 16, 2, 5, 0.3, 700, batch=4, sample_rate=192e9, seed=3)
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    all_out = run_gpu(plan, field)
    for b in range(case.batch):
        one = run_gpu(plan, field[b:b + 1])
        np.testing.assert_array_equal(one[0], all_out[b])


def test_set_coeffs_and_set_ratio_match_fresh_plan():
    import torch
    case = Case(2, 128, 32, 3, 7, 0.3, 1500, sample_rate=128e9, seed=5)
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    taps2 = taps * 1.3 + 0.01
    plan.set_coeffs(taps2.astype(np.float32))
    plan.set_ratio(0.7)
    dev_taps = torch.from_numpy(taps2.astype(np.float32)).cuda()
    a = run_gpu(plan, field)
    plan.set_coeffs(dev_taps)
    b = run_gpu(plan, field)
    case2 = Case(2, 128, 32, 3, 7, 0.7, 1500, sample_rate=128e9, seed=5)
    fresh = run_gpu(make_plan(case2, taps2), field)
    np.testing.assert_array_equal(a, fresh)
    np.testing.assert_array_equal(b, fresh)


def test_alias_and_argument_errors():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    case = Case(1, 64, 16, 1, 3, 0.5, 256)
    plan = make_plan(case, case_taps(case))
    x = torch.zeros(256, 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(cbessfm.CBESSFMError) as ei:
        plan.backpropagate(x, out=x)
    assert ei.value.status == cbessfm.ERR_ALIAS
    with pytest.raises(cbessfm.CBESSFMError) as ei:
        plan.backpropagate_ptr(x.data_ptr() + 8, x.data_ptr() + 8 + 4096, 16, 1, 0)
    assert ei.value.status == cbessfm.ERR_INVALID_ARG


STORAGE_TOL = {1: 3e-3, 2: 3e-3}
STORAGE_CASES = [
    Case(1, 256, 64, 1, 5, 0.5, 2000, storage=1),
    Case(5, 1024, 256, 3, 11, 0.3, 2 * 3840 + 77, sample_rate=640e9, storage=1),
    Case(1, 256, 64, 1, 5, 0.5, 2000, storage=2),
    Case(5, 1024, 256, 3, 11, 0.3, 2 * 3840 + 77, sample_rate=640e9, storage=2),
    Case(3, 64, 16, 2, 7, 0.3, 333, batch=2, sample_rate=192e9, storage=1),
    Case(5, 2048, 512, 2, 11, 0.3, 10240 + 999, sample_rate=640e9, storage=2),
]


@pytest.mark.parametrize("case", STORAGE_CASES, ids=lambda c: f"st{c.storage}_sb{c.n_sb}_np{c.n_fft}"
                         f"_L{c.L}_b{c.batch}")
def test_reduced_precision_storage_matches_oracle(case):
    """FP16 / BF16 storage, FP32 arithmetic: the oracle runs in FP64 on the same quantized input;
    the error is dominated by the rounding of the stored output (relative L2 <= 3e-3)."""
    taps = case_taps(case)
    field = random_field(case)
    plan = make_plan(case, taps)
    got = run_gpu(plan, field)
    q_in = quantize(field, case.storage)
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    for b in range(case.batch):
        want = odbp.dbp_mode_b(q_in[b], p, case.n_fft, case.overlap)
        assert_parity(got[b], want, STORAGE_TOL[case.storage], f"storage{case.storage}/{case}/b{b}")


# Long-haul bound for the complex64 form.  The 1e-5 bound of the FP32 path holds on the plain
# workloads (c1, c2); over 40 strongly nonlinear steps no FP32 chain reaches it.  An FP32 replica
# of the chain whose FFTs are exact (only dispersion, intensity, FIR and rotation rounded to FP32)
# already gives 1.7e-5 on this workload.  With nearest-rounded DFT and twiddle constants the
# kernel measured 3.8e-5 (their norm errors add up coherently over the steps); with the constants
# rounded to keep |w| = 1 it measures 1.7e-5, the replica's floor.  The stated bound leaves room
# for the block sample.
LONG_HAUL_C64_BOUND = 3e-5


@pytest.mark.parametrize("storage,tol", [(0, LONG_HAUL_C64_BOUND), (1, 3e-3), (2, 3e-3)],
                         ids=["complex64", "fp16", "bf16"])
def test_c5_long_haul_sampled_blocks(storage, tol):
    """Long-haul precision workload (5 ch, 40 x 80 km, 2^17 symbols/ch, N' = 2048, 40 steps) in
    the three storage forms: GPU output vs the FP64 oracle on sampled blocks (first, last and
    one interior block), the oracle fed the same storage-rounded input."""
    wl = configs.get_workload("c5_longhaul")
    d, lk, sig = wl.dbp, wl.link, wl.signal
    tx, _ = signals.tx_waveform(wl, wl.launch_dbm[0], seed=wl.seed)
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    taps = signals.random_taps(wl.seed, d.n_st, d.n_sb, d.ntaps, w0, spread=0.2)
    case = Case(d.n_sb, d.n_fft, d.overlap, d.n_st, d.ntaps, d.ratio, sig.n_samples,
                span_length=lk.span_length, n_spans=lk.n_spans, sample_rate=sig.sample_rate,
                storage=storage)
    plan = make_plan(case, taps)
    got = run_gpu(plan, tx[None])[0]
    q_in = quantize(tx[None], storage)[0]
    p = oracle_params(case, taps.astype(np.float32).astype(np.float64))
    nb = plan.n_blocks(case.L)
    want = odbp.dbp_mode_b(q_in, p, d.n_fft, d.overlap, blocks=[0, nb // 2, nb - 1])
    sel = ~np.isnan(want[:, 0])
    assert_parity(got[sel], want[sel], tol, f"c5_longhaul/storage{storage}")


@pytest.fixture(scope="module")
def long_haul_received():
    """A received single-channel DP-16QAM 32 GBd signal after 40 x 80 km (noiseless, oracle SSFM
    with 100 steps per span) -- the input of the precision comparison in SNR terms."""
    lk = configs.Link(n_spans=40, nf_db=None)
    wl = configs.get_workload("c1_tiny").with_(link=lk)
    sig = wl.signal
    tx, syms = signals.tx_waveform(wl, 2.0, seed=21)
    rx = channel.propagate(tx, lk.beta2, lk.gamma, lk.alpha, lk.span_length, lk.n_spans,
                           sig.sample_rate, steps_per_span=100)
    return wl, rx, syms


@pytest.mark.parametrize("storage,max_dq", [(0, 0.02), (1, 0.1), (2, 0.5)],
                         ids=["complex64", "fp16", "bf16"])
def test_long_haul_snr_delta_per_storage(long_haul_received, storage, max_dq):
    """Q-factor (SNR after matched filter, 1 sps and mean-phase removal) of each storage form
    against the FP64 oracle on the same received signal, 40 DBP steps with 5 coupled subbands."""
    wl, rx, syms = long_haul_received
    lk, sig = wl.link, wl.signal
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    n_sb, n_fft, ov, n_st = 5, 512, 128, 40
    taps = signals.random_taps(3, n_st, n_sb, 11, w0 / n_sb, spread=0.1)
    case = Case(n_sb, n_fft, ov, n_st, 11, 0.3, sig.n_samples, span_length=lk.span_length,
                n_spans=lk.n_spans, sample_rate=sig.sample_rate, storage=storage)
    plan = make_plan(case, taps)
    got = run_gpu(plan, rx[None])[0]
    want = odbp.dbp_mode_b(quantize(rx[None], storage)[0],
                           oracle_params(case, taps.astype(np.float32).astype(np.float64)),
                           n_fft, ov)
    p_pol = configs.dbm_to_watt(2.0) / 2
    q = [evaluate.snr_db(evaluate.receive(y, sig.sample_rate, sig.baud, sig.rolloff, 0.0, p_pol),
                         syms[0]) for y in (got, want)]
    rel_l2(got, want, f"long_haul_snr/storage{storage}/dQ={q[0] - q[1]:+.4f}dB/Q={q[1]:.2f}dB")
    assert abs(q[0] - q[1]) <= max_dq, q
