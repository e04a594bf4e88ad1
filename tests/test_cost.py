"""Pins of the complexity model against the numbers the paper prints (Sec. III-D, IV-B)."""
import json
import os

import pytest

from paper_2409_14489_gb300 import cost

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "complexity_sec3d.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_cbessfm_rm_matches_printed_points():
    g = _golden()
    s = g["setup"]
    for pt in g["cbessfm_rm_per_2d"]:
        rm = cost.cbessfm_rm(s["N"], s["N_ov"], s["n"], s["N_sb"], pt["N_st"])
        assert abs(rm - pt["RM"]) <= g["tolerance_rm"], (pt, rm)


def test_edc_rm_matches_printed_value():
    g = _golden()
    s = g["setup"]
    rm = cost.time_domain_rm(s["N"], s["N_ov"], s["n"], N_st=0, N_c=0)
    assert abs(rm - g["edc_rm_per_2d"]) <= g["tolerance_rm"]


def test_single_band_frequency_domain_vs_block_count():
    # With N_sb = 1 the CB-ESSFM count is the ESSFM with frequency-domain NLPR: 4 CFFTs of N,
    # 4 N_st CFFTs of N, N_st + 1 GVDs and N_st NLPRs (Sec. III-D).  Rebuild it from the
    # per-block counts of the text and check the closed form.
    N, N_ov, n, N_st = 4096, 512, 2.0, 3
    import math
    cfft_rm = N * math.log2(N) - 3 * N + 4
    gvd_rm = 6 * N
    nlpr_rm = N * math.log2(N) + N / 2 * (3 * 1 + 13) + 4 * 1
    block_rm = 4 * cfft_rm + 4 * N_st * cfft_rm + (N_st + 1) * gvd_rm + N_st * nlpr_rm
    expect = n * block_rm / (2 * (N - N_ov))
    assert cost.cbessfm_rm(N, N_ov, n, 1, N_st) == pytest.approx(expect, rel=1e-12)


def test_multiband_block_count_rm_and_ra():
    # Same reconstruction with subbands: 4 CFFTs of N, 4 N_sb N_st CFFTs of N' = N / N_sb.
    import math
    N, N_ov, n, N_sb, N_st = 5120, 1280, 2.0, 5, 15
    Np = N // N_sb
    rm_cfft = lambda M: M * math.log2(M) - 3 * M + 4
    ra_cfft = lambda M: 3 * M * math.log2(M) - 3 * M + 4
    nlpr_rm = N * math.log2(Np) + N / 2 * (3 * N_sb + 13) + 4 * N_sb
    nlpr_ra = 3 * N * math.log2(Np) + N / 2 * (5 * N_sb + 11) + 4 * N_sb
    blk_rm = 4 * rm_cfft(N) + 4 * N_sb * N_st * rm_cfft(Np) + (N_st + 1) * 6 * N + N_st * nlpr_rm
    blk_ra = 4 * ra_cfft(N) + 4 * N_sb * N_st * ra_cfft(Np) + (N_st + 1) * 6 * N + N_st * nlpr_ra
    assert cost.cbessfm_rm(N, N_ov, n, N_sb, N_st) == pytest.approx(
        n * blk_rm / (2 * (N - N_ov)), rel=1e-12)
    assert cost.cbessfm_ra(N, N_ov, n, N_sb, N_st) == pytest.approx(
        n * blk_ra / (2 * (N - N_ov)), rel=1e-12)
