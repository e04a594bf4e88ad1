"""Project-written autotuner for the per-job launch parameters of the batched form.

For each job shape (subbands, steps, taps, link, sample rate, storage) it picks:

* the per-subband overlap N'_ov: the dispersion memory of the whole link in samples,
  |beta2| * 2 pi * R * L_link * R (the overlap must cover the channel memory, Sec. III-A), split
  over the subbands and rounded up to a multiple of 16;
* the per-subband FFT size N' in {256, 512, 1024, 2048} (N' > N'_ov, the block fitting one SM):
  ``mode="measure"`` times one launch of each candidate plan on a synthetic block sequence and
  keeps the lowest time per valid sample; ``mode="model"`` uses the paper's operation count per
  2D symbol (Eq. (costRM) plus its RA companion) instead and needs no GPU.

Measured choices are cached in a JSON file (``$CBESSFM_AUTOTUNE_CACHE`` or ``_build/autotune.json``
next to this file), keyed by the job shape.  ``choose_batch`` picks for a whole batch: one N'
per subband count (the batched form's launch groups), the one with the least summed cost over
the group's jobs.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple

from . import cost

CANDIDATE_NFFT = (256, 512, 1024, 2048)
_HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass(frozen=True)
class JobShape:
    n_sb: int
    n_st: int
    ntaps: int
    beta2: float
    link_length: float
    sample_rate: float
    storage: int = 0

    def key(self) -> str:
        return (f"sb{self.n_sb}_st{self.n_st}_t{self.ntaps}_b{self.beta2:.4e}_L{self.link_length:.4e}"
                f"_R{self.sample_rate:.4e}_s{self.storage}")


def memory_samples(shape: JobShape) -> float:
    """Dispersion memory of the link in full-band samples: |beta2| 2 pi R L R."""
    return abs(shape.beta2) * 2.0 * math.pi * shape.sample_rate * shape.link_length * shape.sample_rate


def overlap_for(shape: JobShape) -> int:
    per_sb = memory_samples(shape) / shape.n_sb
    return max(16, int(math.ceil(per_sb / 16.0)) * 16)


# Most subbands the chain kernel takes at each N' (one block's field, exchange arrays and
# intensity rows in one CTA's shared memory); the library's plan_create refuses larger ones.
MAX_BANDS = {2048: 5, 1024: 5, 512: 10, 256: 16}


def _block_fits(n_fft: int, n_sb: int) -> bool:
    """Whether the chain kernel takes N' = n_fft with n_sb subbands in one CTA."""
    return n_sb <= MAX_BANDS.get(n_fft, 16)


def candidates(shape: JobShape):
    ov = overlap_for(shape)
    fitting = [nf for nf in CANDIDATE_NFFT
               if _block_fits(nf, shape.n_sb) and shape.ntaps <= nf // 2]
    if not fitting:
        raise ValueError(f"no block size takes {shape.ntaps} taps with {shape.n_sb} subbands")
    out = [(nf, ov) for nf in fitting if nf > ov]
    if not out:
        # memory longer than any block: the largest block that fits, overlap capped at 3/4 of it
        nf = fitting[-1]
        out.append((nf, min(ov, 3 * nf // 4)))
    return out


def model_cost(shape: JobShape, n_fft: int, overlap: int) -> float:
    """Paper operation count (RM + RA) per valid sample of one block."""
    N, N_ov = shape.n_sb * n_fft, shape.n_sb * overlap
    return cost.cbessfm_flops_per_2d(N, N_ov, 2.0, shape.n_sb, shape.n_st)


class Autotuner:
    def __init__(self, mode: str = "measure", cache_path: Optional[str] = None):
        if mode not in ("measure", "model"):
            raise ValueError(f"mode must be 'measure' or 'model', not {mode!r}")
        self.mode = mode
        self.cache_path = cache_path or os.environ.get(
            "CBESSFM_AUTOTUNE_CACHE", os.path.join(_HERE, "_build", "autotune.json"))
        self.cache: Dict[str, Tuple[int, int]] = {}
        self.times: Dict[str, Dict[Tuple[int, int], float]] = {}
        if mode == "measure" and os.path.exists(self.cache_path):
            try:
                with open(self.cache_path) as f:
                    self.cache = {k: tuple(v) for k, v in json.load(f).items()}
            except (OSError, ValueError):
                self.cache = {}

    def choose(self, shape: JobShape) -> Tuple[int, int]:
        cands = candidates(shape)
        if self.mode == "model" or len(cands) == 1:
            return min(cands, key=lambda c: model_cost(shape, *c))
        k = shape.key()
        if k not in self.cache:
            self.cache[k] = self._measure(shape, cands)
            self._save()
        return self.cache[k]

    def _save(self):
        try:
            os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
        except OSError:
            pass

    def _measure(self, shape: JobShape, cands):
        times = measure_candidates(shape, cands)
        self.times[shape.key()] = times
        return min(times, key=times.get)

    def candidate_costs(self, shape: JobShape) -> Dict[Tuple[int, int], float]:
        """Per-candidate cost per valid sample: measured time (ms, timed once per shape and kept
        for the tuner's life) in measure mode, the paper's operation count in model mode."""
        cands = candidates(shape)
        if self.mode == "model":
            return {c: model_cost(shape, *c) for c in cands}
        k = shape.key()
        if k not in self.times:
            self.times[k] = measure_candidates(shape, cands)
        return self.times[k]

    def choose_batch(self, shapes: Sequence[JobShape],
                     weights: Sequence[float]) -> List[Tuple[int, int]]:
        """(N', N'_ov) for every job of a batch, one N' per subband count and storage type.

        The batched form runs one persistent launch per (N', subbands, storage) group, and a
        group with few work items leaves SMs idle while its last CTAs finish, so choosing each
        job shape's own fastest N' can make the batch slower than a common choice.  Per group of
        jobs that share a subband count and storage type, this picks the N' that minimizes the
        summed cost, each job's cost per valid sample (``candidate_costs``) times its weight
        (its valid samples); each job keeps its own overlap for that N'."""
        if len(shapes) != len(weights):
            raise ValueError("one weight per shape")
        groups: Dict[Tuple[int, int], List[int]] = {}
        for i, sh in enumerate(shapes):
            groups.setdefault((sh.n_sb, sh.storage), []).append(i)
        out: List[Optional[Tuple[int, int]]] = [None] * len(shapes)
        for idx in groups.values():
            costs = [self.candidate_costs(shapes[i]) for i in idx]
            common = set.intersection(*({c[0] for c in cs} for cs in costs))
            if not common:                          # no shared N': each job on its own
                for i, cs in zip(idx, costs):
                    out[i] = min(cs, key=cs.get)
                continue

            def total(nf):
                return sum(weights[i] * next(v for c, v in cs.items() if c[0] == nf)
                           for i, cs in zip(idx, costs))

            best = min(sorted(common), key=total)
            for i, cs in zip(idx, costs):
                out[i] = next(c for c in cs if c[0] == best)
        return out  # type: ignore[return-value]


def measure_candidates(shape: JobShape, cands=None, reps: int = 3) -> Dict[Tuple[int, int], float]:
    """Time per valid sample (ms) of one plain launch of each candidate (N', N'_ov) on a zero
    block sequence long enough to fill the GPU (8 blocks per SM), median-free mean of ``reps``
    launches after two warm-ups."""
    import numpy as np
    import torch
    from . import cbessfm
    cands = candidates(shape) if cands is None else cands
    link = cbessfm.make_link(shape.beta2, shape.link_length, 1, shape.sample_rate)
    taps = np.zeros((shape.n_st, shape.n_sb, shape.n_sb, shape.ntaps), np.float32)
    if shape.n_st:
        taps[..., shape.ntaps // 2] = 1.0
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for nf, ov in cands:
        plan = cbessfm.Plan(link, shape.n_sb, shape.n_st, 0.5, taps, nf, ov, storage=shape.storage)
        V = plan.valid
        L = 8 * n_sm * V                              # enough blocks to fill the GPU
        if shape.storage == 0:
            x = torch.zeros(L, 2, dtype=torch.complex64, device="cuda")
        else:
            dt = torch.float16 if shape.storage == 1 else torch.bfloat16
            x = torch.zeros(L, 4, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(2):
            plan.backpropagate(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.backpropagate(x, y)
        e1.record()
        torch.cuda.synchronize()
        out[(nf, ov)] = e0.elapsed_time(e1) / reps / L                # ms per valid sample
        plan.close()
    return out
