"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This package holds the workload definitions (link, signal and DBP parameters of the five
workloads) and seeded generators of transmitted signals and coefficient taps.  It contains none
of the CB-ESSFM arithmetic: no dispersion step, no nonlinear step, no subband split.  Both the
FP64 oracle (``oracle/``) and the CUDA path consume what it produces.
"""
from .configs import (Link, Signal, DBPParams, Workload, WORKLOADS, get_workload,
                      dbm_to_watt)
from .signals import (qam_symbols, rrc_amplitude, tx_waveform, random_taps, ssfm_delta_taps,
                      effective_length, batch_jobs_c3)

__all__ = [
    "Link", "Signal", "DBPParams", "Workload", "WORKLOADS", "get_workload", "dbm_to_watt",
    "qam_symbols", "rrc_amplitude", "tx_waveform", "random_taps", "ssfm_delta_taps",
    "effective_length", "batch_jobs_c3",
]
