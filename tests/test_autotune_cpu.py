"""Host logic of the batched form's autotuner (paper_2409_14489_gb300/autotune.py), on CPU: the
overlap covers the link's dispersion memory, the candidate list respects the block limits, the
cost model picks the candidate with the lowest paper operation count per valid sample, and a
cached measurement is reused without touching a GPU."""
import json
import math

import pytest

from paper_2409_14489_gb300 import autotune, cost


def _shape(n_sb=1, n_st=1, ntaps=5, L=80e3, R=64e9):
    return autotune.JobShape(n_sb, n_st, ntaps, -21.7e-27, L, R)


def test_memory_and_overlap_follow_the_dispersion_spread():
    s = _shape()
    # |beta2| 2 pi R^2 L: about 44.7 samples for 80 km at 64 GS/s
    want = 21.7e-27 * 2 * math.pi * 64e9 ** 2 * 80e3
    assert autotune.memory_samples(s) == pytest.approx(want, rel=1e-12)
    assert autotune.overlap_for(s) == 48                    # rounded up to a multiple of 16
    assert autotune.overlap_for(_shape(n_sb=3)) == 16       # 14.9 per subband
    assert autotune.overlap_for(_shape(n_sb=5)) == 16       # 8.9, at least 16
    assert autotune.overlap_for(_shape(L=1200e3)) == 672    # 15 spans: 670.5 -> 672
    for n_sb in (1, 2, 3, 5):
        for L in (80e3, 400e3, 1200e3):
            ov = autotune.overlap_for(_shape(n_sb=n_sb, L=L))
            assert ov % 16 == 0 and ov * n_sb >= autotune.memory_samples(_shape(n_sb=n_sb, L=L))


def test_candidates_respect_overlap_taps_and_block_limits():
    s = _shape(L=1200e3)                                     # overlap 672
    nfs = [nf for nf, _ in autotune.candidates(s)]
    assert nfs == [1024, 2048]
    assert all(ov == 672 for _, ov in autotune.candidates(s))
    assert [nf for nf, _ in autotune.candidates(_shape(ntaps=601))] == [2048]
    assert 2048 not in [nf for nf, _ in autotune.candidates(_shape(n_sb=6))]
    # memory longer than any block: the largest block that fits, overlap capped at 3/4 of it
    assert autotune.candidates(_shape(L=5000e3)) == [(2048, 1536)]
    assert autotune.candidates(_shape(n_sb=6, L=50000e3)) == [(512, 384)]
    assert autotune.candidates(_shape(n_sb=12, L=50000e3)) == [(256, 192)]
    with pytest.raises(ValueError, match="taps"):
        autotune.candidates(_shape(ntaps=1025))
    with pytest.raises(ValueError, match="mode"):
        autotune.Autotuner("fastest")


def test_model_mode_picks_the_cheapest_candidate():
    tuner = autotune.Autotuner("model")
    for n_sb in (1, 3, 5):
        for n_st in (1, 4, 15):
            for L in (80e3, 800e3):
                s = _shape(n_sb=n_sb, n_st=n_st, L=L, R=64e9 * n_sb)
                nf, ov = tuner.choose(s)
                costs = {c: autotune.model_cost(s, *c) for c in autotune.candidates(s)}
                assert costs[(nf, ov)] == min(costs.values())
                N, N_ov = n_sb * nf, n_sb * ov
                assert autotune.model_cost(s, nf, ov) == cost.cbessfm_flops_per_2d(
                    N, N_ov, 2.0, n_sb, n_st)


def test_measured_choice_is_read_back_from_the_cache(tmp_path):
    s = _shape(n_sb=3, n_st=4, L=80e3, R=192e9)              # overlap 144: four candidates
    assert len(autotune.candidates(s)) == 4
    path = tmp_path / "autotune.json"
    path.write_text(json.dumps({s.key(): [512, 144]}))
    tuner = autotune.Autotuner("measure", cache_path=str(path))
    assert tuner.choose(s) == (512, 144)                    # no launch needed for a cached shape
    assert s.key() != _shape(n_sb=3, n_st=4, L=80e3, R=192e9, ntaps=7).key()


def test_block_limits_agree_with_the_library():
    """The tuner's subband limits per N' are exactly the plans the library accepts.  plan_create
    checks threads and shared memory before touching the device, so without a GPU an accepted
    plan fails later with CBESSFM_ERR_CUDA and a refused one returns CBESSFM_ERR_UNSUPPORTED."""
    import ctypes
    import numpy as np
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_14489_gb300 import cbessfm as cb
    L = cb.lib()
    link = cb.make_link(-21.7e-27, 80e3, 1, 64e9)
    for nf in autotune.CANDIDATE_NFFT:
        for n_sb in range(1, 17):
            taps = np.zeros((1, n_sb, n_sb, 11), np.float32)
            h = ctypes.c_void_p()
            st = L.cbessfm_plan_create(ctypes.byref(link), n_sb, 1, 0.5,
                                       taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 11,
                                       nf, nf // 4, 0, ctypes.byref(h))
            if st == cb.OK:
                L.cbessfm_plan_destroy(h)
            assert st in (cb.OK, cb.ERR_CUDA, cb.ERR_UNSUPPORTED), (nf, n_sb, st)
            assert (st != cb.ERR_UNSUPPORTED) == autotune._block_fits(nf, n_sb), (nf, n_sb)


def test_batch_choice_is_one_block_size_per_subband_count(tmp_path):
    """choose_batch: jobs sharing a subband count get one N' (one persistent launch), the one
    with the least weighted summed cost, even where a job's own fastest N' differs; each job
    keeps its own overlap.  Measured costs are planted, so no GPU is touched."""
    tuner = autotune.Autotuner("measure", cache_path=str(tmp_path / "t.json"))
    a = _shape(n_sb=3, n_st=1, L=80e3, R=192e9)
    b = _shape(n_sb=3, n_st=15, L=80e3, R=192e9)
    c = _shape(n_sb=1, n_st=4, L=80e3, R=64e9)
    ov3 = autotune.overlap_for(a)
    ov1 = autotune.overlap_for(c)
    # a alone prefers 512, b alone prefers 1024; with b weighted 3x, 1024 wins the group:
    # 1 x 1.00 + 3 x 1.00 = 4.00 (1024) against 1 x 0.95 + 3 x 1.10 = 4.25 (512)
    tuner.times[a.key()] = {(256, ov3): 1.30, (512, ov3): 0.95, (1024, ov3): 1.00, (2048, ov3): 1.40}
    tuner.times[b.key()] = {(256, ov3): 1.20, (512, ov3): 1.10, (1024, ov3): 1.00, (2048, ov3): 1.30}
    tuner.times[c.key()] = {(nf, ov1): t for nf, t in ((256, 2.0), (512, 1.0), (1024, 1.2),
                                                       (2048, 1.5))}
    got = tuner.choose_batch([a, b, c, b], [1.0, 1.5, 7.0, 1.5])
    assert got == [(1024, ov3), (1024, ov3), (512, ov1), (1024, ov3)]
    # with a weighted up instead, the group moves to a's choice
    assert tuner.choose_batch([a, b], [10.0, 1.0]) == [(512, ov3), (512, ov3)]
    with pytest.raises(ValueError):
        tuner.choose_batch([a], [1.0, 2.0])


def test_batch_choice_in_model_mode_minimizes_the_summed_operation_count():
    tuner = autotune.Autotuner("model")
    shapes = [_shape(n_sb=5, n_st=n, L=80e3, R=320e9) for n in (1, 4, 15)]
    weights = [3.0, 1.0, 2.0]
    got = tuner.choose_batch(shapes, weights)
    assert len({nf for nf, _ in got}) == 1
    nfs = {c[0] for c in autotune.candidates(shapes[0])}

    def total(nf):
        return sum(w * next(autotune.model_cost(s, *c) for c in autotune.candidates(s)
                            if c[0] == nf) for s, w in zip(shapes, weights))

    assert total(got[0][0]) == min(total(nf) for nf in nfs)
