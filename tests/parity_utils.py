"""Helpers shared by the GPU parity tests: one case description feeds both the CUDA plan and the
FP64 oracle with identical parameters and inputs."""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import numpy as np

from oracle import dbp as odbp
from synth import signals


@dataclass
class Case:
    n_sb: int
    n_fft: int
    overlap: int
    n_st: int
    ntaps: int
    ratio: float
    L: int
    batch: int = 1
    beta2: float = -21.7e-27
    span_length: float = 80e3
    n_spans: int = 1
    sample_rate: float = 64e9
    tap_scale: float = 0.1
    field_scale: float = 1.0
    seed: int = 0
    storage: int = 0          # 0 complex64, 1 fp16 x 4, 2 bf16 x 4

    @property
    def link_length(self) -> float:
        return self.span_length * self.n_spans


def random_field(case: Case) -> np.ndarray:
    rng = np.random.default_rng(case.seed)
    shape = (case.batch, case.L, 2)
    f = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)
    return (case.field_scale * f).astype(np.complex128)


def case_taps(case: Case) -> np.ndarray:
    return signals.random_taps(case.seed + 17, case.n_st, case.n_sb, case.ntaps, case.tap_scale,
                               spread=0.3)


def oracle_params(case: Case, taps: np.ndarray) -> odbp.ChainParams:
    return odbp.ChainParams(beta2=case.beta2, sample_rate=case.sample_rate,
                            link_length=case.link_length, n_sb=case.n_sb, ratio=case.ratio,
                            taps=np.asarray(taps, dtype=np.float64))


def make_plan(case: Case, taps: np.ndarray):
    from paper_2409_14489_gb300 import cbessfm
    link = cbessfm.make_link(case.beta2, case.span_length, case.n_spans, case.sample_rate)
    return cbessfm.Plan(link, case.n_sb, case.n_st, case.ratio,
                        np.asarray(taps, dtype=np.float32), case.n_fft, case.overlap,
                        storage=case.storage)


def to_storage(field: np.ndarray, storage: int):
    """complex (..., L, 2) -> a CUDA tensor in the plan's storage layout."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(field.astype(np.complex64))).cuda()
    if storage == 0:
        return x
    dt = torch.float16 if storage == 1 else torch.bfloat16
    return torch.view_as_real(x).reshape(*x.shape[:-1], 4).to(dt).contiguous()


def from_storage(y, storage: int) -> np.ndarray:
    import torch
    if storage == 0:
        return y.cpu().numpy().astype(np.complex128)
    r = y.float().reshape(*y.shape[:-1], 2, 2)
    return torch.view_as_complex(r.contiguous()).cpu().numpy().astype(np.complex128)


def quantize(field: np.ndarray, storage: int) -> np.ndarray:
    """The input as the GPU sees it after storage rounding (for the oracle)."""
    return from_storage(to_storage(field, storage), storage)


def run_gpu(plan, field: np.ndarray) -> np.ndarray:
    import torch
    x = to_storage(field, plan.storage)
    y = plan.backpropagate(x)
    torch.cuda.synchronize()
    return from_storage(y, plan.storage)


def rel_l2(a: np.ndarray, b: np.ndarray, name: str = "") -> float:
    """Relative L2 error ||a - b|| / ||b||; logged to $CBESSFM_PARITY_LOG (JSON lines) if set."""
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    log = os.environ.get("CBESSFM_PARITY_LOG")
    if log and name:
        with open(log, "a") as f:
            f.write(json.dumps({"case": name, "rel_l2": err}) + "\n")
    return err


# Per-sample bound beside the relative L2 error: a defect confined to a few samples (one block
# edge, one subband) moves the L2 norm little but shows in the largest sample error.  Every
# sample's error must stay within PEAK_FACTOR x tol of the oracle's RMS sample magnitude.
PEAK_FACTOR = 10.0


def peak_rel(a: np.ndarray, b: np.ndarray) -> float:
    """max_k |a_k - b_k| / rms(b): the largest sample error against the RMS sample magnitude."""
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    return float(d / np.sqrt(np.mean(np.abs(np.asarray(b)) ** 2)))


def assert_parity(got: np.ndarray, want: np.ndarray, tol: float, name: str = "") -> float:
    """rel-L2 <= tol and every sample within PEAK_FACTOR * tol * rms(want); returns the rel-L2."""
    err = rel_l2(got, want, name)
    peak = peak_rel(got, want)
    log = os.environ.get("CBESSFM_PARITY_LOG")
    if log and name:
        with open(log, "a") as f:
            f.write(json.dumps({"case": name + "/peak", "peak_rel": peak}) + "\n")
    assert err <= tol, (name, err, tol)
    assert peak <= PEAK_FACTOR * tol, (name, "peak", peak, PEAK_FACTOR * tol)
    return err
