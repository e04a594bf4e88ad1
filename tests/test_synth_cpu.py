"""The synthetic workloads (synth/) match the recipe they stand for: shapes, rates and DBP
parameters of the five configurations, the c3 job list's distributions, the transmitter's unit
symbol energy and launch power, and seeded reproducibility."""
import math

import numpy as np
import pytest

from synth import configs, signals


def test_workload_shapes_and_rates():
    c1 = configs.get_workload("c1_tiny")
    assert (c1.signal.n_ch, c1.signal.baud, c1.signal.qam, c1.signal.sample_rate) == (1, 32e9, 16, 64e9)
    assert c1.signal.n_samples == 2 * 2 ** 12 and c1.link.n_spans == 1
    assert (c1.dbp.n_sb, c1.dbp.n_st, c1.dbp.ntaps, c1.dbp.n_fft, c1.dbp.overlap) == (1, 1, 5, 256, 64)
    c2 = configs.get_workload("c2_wdm15")
    assert (c2.signal.n_ch, c2.signal.baud, c2.signal.qam, c2.signal.ch_spacing) == (5, 64e9, 64, 100e9)
    assert c2.signal.sample_rate == 2 * 5 * 64e9 and c2.signal.n_samples == 655360
    assert c2.link.n_spans == 15 and c2.link.nf_db == 5.0
    assert list(c2.launch_dbm) == [-2.0, -1.0, 0.0, 1.0, 2.0, 3.0, 4.0]
    assert (c2.dbp.n_sb, c2.dbp.n_st, c2.dbp.ratio, c2.dbp.ntaps, c2.dbp.n_fft, c2.dbp.overlap) == \
        (5, 15, 0.3, 11, 1024, 256)
    c4 = configs.get_workload("c4_adjoint")
    assert c4.batch == 32 and c4.signal.n_sym == 2 ** 15 and c4.link.n_spans == 15
    assert (c4.dbp.n_sb, c4.dbp.n_st, c4.dbp.ntaps) == (5, 15, 11)
    c5 = configs.get_workload("c5_longhaul")
    assert c5.link.n_spans == 40 and c5.signal.n_sym == 2 ** 17 and c5.dbp.n_fft == 2048
    assert c5.dbp.n_st == 40 and c5.signal.n_samples == 1310720


def test_c3_job_list_distributions():
    jobs = signals.batch_jobs_c3(3)
    assert len(jobs) == 256
    n_sym = np.array([j["n_samples"] / 2 for j in jobs])
    assert n_sym.min() >= 2 ** 12 - 32 and n_sym.max() <= 2 ** 17
    assert all(j["n_samples"] % 64 == 0 for j in jobs)
    # log-uniform: log2 of the lengths spreads evenly over [12, 17]
    lg = np.log2(n_sym)
    assert abs(np.mean(lg) - 14.5) < 0.3 and np.std(lg) == pytest.approx(5 / math.sqrt(12), rel=0.15)
    assert {j["n_st"] for j in jobs} == {1, 2, 4, 8, 15}
    assert {j["n_sb"] for j in jobs} == {1, 3, 5}
    assert signals.batch_jobs_c3(3) == jobs                      # seeded
    assert signals.batch_jobs_c3(4) != jobs


def test_transmitter_power_and_symbol_energy():
    wl = configs.get_workload("c2_wdm15")
    f, syms = signals.tx_waveform(wl, 1.0, seed=2)
    assert f.shape == (wl.signal.n_samples, 2) and syms.shape == (5, wl.signal.n_sym, 2)
    # unit mean symbol energy of square 64-QAM, per polarization and channel
    assert np.mean(np.abs(syms) ** 2) == pytest.approx(1.0, rel=0.02)
    # average power: 5 channels at +1 dBm each (both polarizations together)
    p_tot = np.mean(np.sum(np.abs(f) ** 2, axis=1))
    assert p_tot == pytest.approx(5 * configs.dbm_to_watt(1.0), rel=0.03)
    f2, _ = signals.tx_waveform(wl, 1.0, seed=2)
    assert np.array_equal(f, f2)
