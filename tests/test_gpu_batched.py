"""Batched form (cbessfm_batch_*): a persistent launch per (N', subbands, storage) group over a
work list of uneven jobs must reproduce the plain per-job launches bit for bit (same per-block
arithmetic), also when captured in a CUDA graph and replayed, and stay within the oracle
tolerance."""
import numpy as np
import pytest

from oracle import dbp as odbp
from synth import configs, signals

from parity_utils import Case, random_field, case_taps, oracle_params, make_plan, rel_l2, \
    to_storage, from_storage

pytestmark = pytest.mark.gpu


def _jobs(cases):
    import torch
    jobs = []
    for c in cases:
        taps = case_taps(c)
        plan = make_plan(c, taps)
        x = to_storage(random_field(c)[0], c.storage)
        y = torch.full_like(x, float("nan")) if c.storage == 0 else torch.empty_like(x)
        jobs.append((c, taps, plan, x, y))
    return jobs


MIXED = [
    Case(1, 256, 64, 1, 5, 0.5, 8192, seed=1),
    Case(1, 256, 64, 4, 5, 0.5, 3001, seed=2),
    Case(3, 256, 16, 2, 5, 0.3, 20000, sample_rate=192e9, seed=3),
    Case(5, 1024, 256, 15, 11, 0.3, 40000, sample_rate=640e9, seed=4),
    Case(5, 1024, 256, 3, 11, 0.3, 9000, sample_rate=640e9, seed=5),
    Case(3, 256, 16, 8, 7, 0.12, 777, sample_rate=192e9, seed=6),
    Case(2, 2048, 512, 2, 11, 0.3, 12345, sample_rate=128e9, seed=7),
    Case(1, 64, 16, 2, 3, 0.5, 50, seed=8),                        # shorter than one block
    Case(5, 1024, 256, 2, 11, 0.3, 7000, sample_rate=640e9, seed=9, storage=1),
]


def test_batched_matches_plain_launches_bitwise():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    jobs = _jobs(MIXED)
    batch = cbessfm.Batch([(plan, x, y) for _, _, plan, x, y in jobs])
    info = batch.info()
    assert info["groups"] == 6
    batch.run()
    torch.cuda.synchronize()
    for c, taps, plan, x, y in jobs:
        ref = plan.backpropagate(x)
        torch.cuda.synchronize()
        assert torch.equal(y, ref), c
        assert plan.status() == 0


def test_batched_16bit_storage_mixed_staging_bitwise():
    """One persistent launch over FP16 jobs whose blocks are staged by bulk copies (even length
    and start) and by plain loads (odd length or odd start), interleaved on the same CTAs: the
    staging mbarrier's phases stay in step, and each job equals its plain launch."""
    import torch
    from paper_2409_14489_gb300 import cbessfm
    # overlap 16: even block starts (bulk copies for an even length, a mix for an odd one);
    # overlap 18: odd starts (plain loads)
    cases = [Case(3, 256, ov, 2, 5, 0.3, n, sample_rate=192e9, seed=20 + k, storage=st)
             for k, (n, st, ov) in enumerate([(4000, 1, 16), (4001, 1, 16), (6000, 1, 18),
                                              (2999, 1, 16), (5000, 2, 16), (5001, 2, 18)])]
    jobs = _jobs(cases)
    batch = cbessfm.Batch([(plan, x, y) for _, _, plan, x, y in jobs])
    batch.run()
    torch.cuda.synchronize()
    for c, taps, plan, x, y in jobs:
        ref = plan.backpropagate(x)
        torch.cuda.synchronize()
        assert torch.equal(y, ref), c
        assert plan.status() == 0


def test_batched_job_against_oracle():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    jobs = _jobs(MIXED[:4])
    batch = cbessfm.Batch([(plan, x, y) for _, _, plan, x, y in jobs])
    batch.run()
    torch.cuda.synchronize()
    for c, taps, plan, x, y in jobs:
        got = from_storage(y, c.storage)
        want = odbp.dbp_mode_b(from_storage(x, c.storage), oracle_params(
            c, taps.astype(np.float32).astype(np.float64)), c.n_fft, c.overlap)
        assert rel_l2(got, want, f"batched/{c}") <= 1e-5


def test_batched_graph_replay_follows_buffers():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    jobs = _jobs(MIXED[2:6])
    batch = cbessfm.Batch([(plan, x, y) for _, _, plan, x, y in jobs])
    graph = batch.capture()
    graph.replay()
    torch.cuda.synchronize()
    first = [y.clone() for *_, y in jobs]
    for c, taps, plan, x, y in jobs:
        x.mul_(0.5)                                  # new data in the same buffers
    graph.replay()
    torch.cuda.synchronize()
    for (c, taps, plan, x, y), y0 in zip(jobs, first):
        assert not torch.equal(y, y0)
        assert torch.equal(y, plan.backpropagate(x)), c
    graph.replay()
    torch.cuda.synchronize()
    for (c, taps, plan, x, y) in jobs:
        assert torch.equal(y, plan.backpropagate(x))


def c3_jobs(tuner_mode="model"):
    """The batched workload: 256 uneven realizations of the c1 signal model (32 GBd DP-16QAM,
    2 samples/symbol, 1 x 80 km), steps in {1,2,4,8,15}, subbands in {1,3,5}; N' and overlap
    from the autotuner."""
    from paper_2409_14489_gb300 import autotune
    wl = configs.get_workload("c3_batched")
    lk, sig = wl.link, wl.signal
    tuner = autotune.Autotuner(tuner_mode)
    out = []
    for k, jb in enumerate(signals.batch_jobs_c3(wl.seed)):
        shape = autotune.JobShape(jb["n_sb"], jb["n_st"], wl.dbp.ntaps, lk.beta2, lk.length,
                                  sig.sample_rate)
        n_fft, ov = tuner.choose(shape)
        case = Case(jb["n_sb"], n_fft, ov, jb["n_st"], wl.dbp.ntaps, wl.dbp.ratio,
                    jb["n_samples"], sample_rate=sig.sample_rate, seed=jb["seed"] % 100000)
        out.append(case)
    return out


def test_c3_batched_workload_matches_plain_and_sampled_oracle():
    import torch
    from paper_2409_14489_gb300 import cbessfm
    wl = configs.get_workload("c3_batched")
    lk = wl.link
    w0 = lk.gamma * signals.effective_length(lk.alpha, lk.span_length)
    cases = c3_jobs()
    jobs = []
    rng = np.random.default_rng(3)
    for c in cases:
        taps = signals.random_taps(c.seed, c.n_st, c.n_sb, c.ntaps, w0 / c.n_st, spread=0.2)
        plan = make_plan(c, taps)
        f = 0.03 * (rng.standard_normal((c.L, 2)) + 1j * rng.standard_normal((c.L, 2)))
        x = to_storage(f, 0)
        jobs.append((c, taps, plan, x, torch.empty_like(x)))
    batch = cbessfm.Batch([(plan, x, y) for _, _, plan, x, y in jobs])
    graph = batch.capture()
    graph.replay()
    torch.cuda.synchronize()
    for k, (c, taps, plan, x, y) in enumerate(jobs):
        assert torch.equal(y, plan.backpropagate(x)), k
    for k in (0, 17, 101, 255):
        c, taps, plan, x, y = jobs[k]
        want = odbp.dbp_mode_b(from_storage(x, 0), oracle_params(
            c, taps.astype(np.float32).astype(np.float64)), c.n_fft, c.overlap, blocks=[0])
        sel = ~np.isnan(want[:, 0])
        assert rel_l2(from_storage(y, 0)[sel], want[sel], f"c3/job{k}") <= 1e-5
