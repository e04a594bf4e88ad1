"""Complexity model of the paper (Sec. III-D), used for algorithmic flop counts.

Counting rules of the paper: a complex multiplication costs 3 RM + 5 RA (3 RA with a known
multiplier, 4 RA on average when two share a multiplier, 2 RM with a real multiplier), a CFFT
of size N costs N log2 N - 3N + 4 RM and 3N log2 N - 3N + 4 RA (split radix), an RFFT about
half of that, and the complex exponential is not counted.

* ``cbessfm_rm`` / ``cbessfm_ra``: Eq. (costRM) and its RA companion, per 2D symbol.
* ``time_domain_rm`` / ``time_domain_ra``: Eqs. (compl_RM_time), (compl_RA_time) for the
  time-domain ESSFM; N_c = 0 gives SSFM/OSSFM, N_st = 0 gives EDC.

The flop count used for the roofline is RM + RA (each one floating-point operation).
"""
from __future__ import annotations

import math


def cbessfm_rm(N: int, N_ov: int, n: float, N_sb: int, N_st: int) -> float:
    """Real multiplications per 2D symbol of the CB-ESSFM (Eq. (costRM))."""
    body = ((5 * N_st + 4) * math.log2(N / N_sb) + N_st * (3 * N_sb + 1) / 2.0
            + 4 * math.log2(N_sb) - 6 + (20 * N_sb * N_st + 16) / N)
    return n / 2.0 * N / (N - N_ov) * body


def cbessfm_ra(N: int, N_ov: int, n: float, N_sb: int, N_st: int) -> float:
    """Real additions per 2D symbol of the CB-ESSFM (companion of Eq. (costRM))."""
    body = ((15 * N_st + 12) * math.log2(N / N_sb) + N_st * (5 * N_sb - 1) / 2.0
            + 12 * math.log2(N_sb) - 6 + (20 * N_sb * N_st + 16) / N)
    return n / 2.0 * N / (N - N_ov) * body


def time_domain_rm(N: int, N_ov: int, n: float, N_st: int, N_c: int) -> float:
    """Real multiplications per 2D symbol of the time-domain ESSFM (Eq. (compl_RM_time))."""
    body = (N_st + 1) * (4 * math.log2(N) - 6 + 16.0 / N) + N_st * (11 + N_c)
    return n / 2.0 * N / (N - N_ov) * body


def time_domain_ra(N: int, N_ov: int, n: float, N_st: int, N_c: int) -> float:
    """Real additions per 2D symbol of the time-domain ESSFM (Eq. (compl_RA_time))."""
    body = (N_st + 1) * (12 * math.log2(N) - 6 + 16.0 / N) + N_st * (11 + 2 * N_c)
    return n / 2.0 * N / (N - N_ov) * body


def cbessfm_flops_per_2d(N: int, N_ov: int, n: float, N_sb: int, N_st: int) -> float:
    """Algorithmic floating-point operations (RM + RA) per 2D symbol."""
    return cbessfm_rm(N, N_ov, n, N_sb, N_st) + cbessfm_ra(N, N_ov, n, N_sb, N_st)


def sym2d_per_sample(n: float) -> float:
    """Each 4D sample at n samples per (4D) symbol carries 2/n 2D symbols."""
    return 2.0 / n
