"""Workload definitions: fiber link, transmitted signal and DBP parameters (SI units).

The five workloads mirror the shapes of the paper's simulation setup (Sec. IV-A: 15 x 80 km
SMF, 5 WDM channels at 100 GHz, dual-polarization QAM with RRC pulses) at the sizes used for
parity tests and benchmarks:

* ``c1_tiny``       single channel DP-16QAM 32 GBd, 1 x 80 km, 1 DBP step, 1 subband.
* ``c2_wdm15``      5 ch DP-64QAM 64 GBd, 15 x 80 km, 5 subbands, 15 asymmetric steps (rho=0.3).
* ``c3_batched``    256 uneven realizations of the c1 signal model (job list in signals.py).
* ``c4_adjoint``    32 realizations x 2^15 symbols of the c1 signal model over 15 x 80 km.
* ``c5_longhaul``   5 ch DP-64QAM 64 GBd, 40 x 80 km, 40 steps, 5 subbands, N'=2048.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple


def dbm_to_watt(p_dbm: float) -> float:
    return 1e-3 * 10.0 ** (p_dbm / 10.0)


@dataclass(frozen=True)
class Link:
    beta2: float = -21.7e-27        # s^2/m  (-21.7 ps^2/km)
    gamma: float = 1.3e-3           # 1/(W m) (1.3 /W/km)
    alpha_db_km: float = 0.2        # dB/km power attenuation
    span_length: float = 80e3       # m
    n_spans: int = 1
    nf_db: Optional[float] = None   # EDFA noise figure; None = noiseless ideal EDFA

    @property
    def alpha(self) -> float:
        """Power attenuation coefficient in 1/m."""
        return self.alpha_db_km / (10.0 * math.log10(math.e)) / 1e3

    @property
    def length(self) -> float:
        return self.span_length * self.n_spans


@dataclass(frozen=True)
class Signal:
    n_ch: int = 1
    baud: float = 32e9              # symbols/s per channel
    ch_spacing: float = 100e9       # Hz
    qam: int = 16                   # square QAM order per polarization
    rolloff: float = 0.1
    n_sym: int = 2 ** 12            # symbols per channel and polarization
    sample_rate: float = 64e9       # full-band sampling rate R

    @property
    def n_samples(self) -> int:
        """Samples of one period of the field."""
        sps = self.sample_rate / self.baud
        n = self.n_sym * sps
        assert abs(n - round(n)) < 1e-9
        return int(round(n))

    @property
    def sym2d_per_realization(self) -> int:
        """2D symbols = 2 polarizations x channels x symbols."""
        return 2 * self.n_ch * self.n_sym


@dataclass(frozen=True)
class DBPParams:
    n_sb: int = 1                   # subbands N_sb
    n_st: int = 1                   # steps N_st
    ratio: float = 0.5              # splitting ratio rho
    ntaps: int = 5                  # 2 N_c + 1
    n_fft: int = 256                # N' (per subband)
    overlap: int = 64               # N'_ov (per subband)

    @property
    def n_block(self) -> int:
        return self.n_sb * self.n_fft

    @property
    def n_ov_total(self) -> int:
        return self.n_sb * self.overlap


@dataclass(frozen=True)
class Workload:
    name: str
    link: Link
    signal: Signal
    dbp: DBPParams
    launch_dbm: Tuple[float, ...] = (0.0,)   # per channel, one realization each
    seed: int = 1

    @property
    def batch(self) -> int:
        return len(self.launch_dbm)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


_C1 = Workload(
    name="c1_tiny",
    link=Link(n_spans=1, nf_db=None),
    signal=Signal(n_ch=1, baud=32e9, qam=16, rolloff=0.1, n_sym=2 ** 12, sample_rate=64e9),
    dbp=DBPParams(n_sb=1, n_st=1, ratio=0.5, ntaps=5, n_fft=256, overlap=64),
    launch_dbm=(0.0,), seed=1)

_C2 = Workload(
    name="c2_wdm15",
    link=Link(n_spans=15, nf_db=5.0),
    signal=Signal(n_ch=5, baud=64e9, ch_spacing=100e9, qam=64, rolloff=0.05, n_sym=2 ** 16,
                  sample_rate=640e9),
    dbp=DBPParams(n_sb=5, n_st=15, ratio=0.3, ntaps=11, n_fft=1024, overlap=256),
    launch_dbm=(-2.0, -1.0, 0.0, 1.0, 2.0, 3.0, 4.0), seed=0)

_C4 = Workload(
    name="c4_adjoint",
    link=Link(n_spans=15, nf_db=None),
    signal=Signal(n_ch=1, baud=32e9, qam=16, rolloff=0.1, n_sym=2 ** 15, sample_rate=64e9),
    dbp=DBPParams(n_sb=5, n_st=15, ratio=0.3, ntaps=11, n_fft=1024, overlap=256),
    launch_dbm=(0.0,) * 32, seed=4)

_C5 = Workload(
    name="c5_longhaul",
    link=Link(n_spans=40, nf_db=5.0),
    signal=Signal(n_ch=5, baud=64e9, ch_spacing=100e9, qam=64, rolloff=0.05, n_sym=2 ** 17,
                  sample_rate=640e9),
    dbp=DBPParams(n_sb=5, n_st=40, ratio=0.3, ntaps=11, n_fft=2048, overlap=512),
    launch_dbm=(2.0,), seed=5)

_C3 = Workload(
    name="c3_batched",
    link=Link(n_spans=1, nf_db=None),
    signal=Signal(n_ch=1, baud=32e9, qam=16, rolloff=0.1, n_sym=2 ** 12, sample_rate=64e9),
    dbp=DBPParams(n_sb=1, n_st=1, ratio=0.5, ntaps=5, n_fft=256, overlap=64),
    launch_dbm=(0.0,), seed=3)

WORKLOADS = {w.name: w for w in (_C1, _C2, _C3, _C4, _C5)}


def get_workload(name: str) -> Workload:
    return WORKLOADS[name]
