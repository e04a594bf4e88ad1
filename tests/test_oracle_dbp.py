"""Pins of the FP64 oracle chain (oracle.dbp) against closed forms, invariants and independent
textbook algorithms.  None of these re-types the oracle's own code path:

* FFT primitive vs brute-force DFT (the oracle uses numpy's FFT as a library step).
* Subband DEMUX: exact partition of the band, inverse MUX, unit-tone normalization, Parseval, and
  reconstruction of the full-band samples from the subband samples (Eq. (subband-division)).
* Linear chain (all taps zero): equals one closed-form dispersion exp(+j beta2 w^2 Z / 2) over
  the whole link for every subband count, splitting ratio and step count (Sec. III-A, III-C).
* beta2 = 0, one band, centre-tap-only filters: the exact SPM rotation u exp(j sum phi |u|^2).
* Energy per step and pointwise intensity are preserved by the NLPR (Sec. III-A, Fig. 3).
* The time-domain MIMO filter equals the paper's frequency-domain MIMO implementation (Fig. 3).
* One band with centre-tap-only filters equals an independently written asymmetric SSFM.
* Frequency-shift equivariance with circulant coupling taps and beta2 = 0 (checks the DEMUX
  index map and the XPM coupling indices).
* Overlap-and-save: circular-shift equivariance by V samples, and agreement with the whole-
  sequence chain when the overlap covers the channel memory.
* Chain inversion: every operator of the chain is invertible (GVD is unitary, the rotation keeps
  |u|^2 so its phase can be recomputed from its output), and the chain with -beta2, the ratio
  1 - rho and the negated taps in reverse step order undoes it.
"""
import math

import numpy as np
import pytest

from oracle import dbp
from synth import configs, signals

RNG = np.random.default_rng(1234)


def _rand_field(L, rng=RNG, scale=1.0):
    return scale * (rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2))) / math.sqrt(2)


# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 16, 20, 40, 48, 64])
def test_fft_primitive_matches_bruteforce_dft(n):
    x = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    k = np.arange(n)
    dft = np.exp(-2j * math.pi * np.outer(k, k) / n) @ x
    np.testing.assert_allclose(np.fft.fft(x), dft, rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(np.fft.ifft(dft), x, rtol=0, atol=1e-12 * max(1, n))


# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n_sb,n_sub", [(1, 16), (2, 8), (3, 16), (5, 32), (4, 64)])
def test_subbands_partition_band_and_mux_inverts_demux(n_sb, n_sub):
    N = n_sb * n_sub
    K, b = dbp.subband_bins(N, n_sb)
    assert sorted(K.reshape(-1).tolist()) == list(range(N))
    assert sorted(b.reshape(-1).tolist()) == list(range(-N // 2, N // 2))
    # subband i owns the i-th contiguous slice of [-N/2, N/2)
    for i in range(n_sb):
        assert b[i].min() == -N // 2 + i * n_sub and b[i].max() == -N // 2 + (i + 1) * n_sub - 1
    U = RNG.standard_normal((N, 2)) + 1j * RNG.standard_normal((N, 2))
    np.testing.assert_array_equal(dbp.mux(dbp.demux(U, n_sb)), U)


@pytest.mark.parametrize("n_sb,n_sub", [(1, 16), (2, 16), (3, 32), (5, 32)])
def test_subband_samples_unit_tone_parseval_and_reconstruction(n_sb, n_sub):
    N = n_sb * n_sub
    n = np.arange(N)
    _, b = dbp.subband_bins(N, n_sb)
    for i in range(n_sb):
        c_i = -N // 2 + i * n_sub + n_sub // 2
        tone = np.exp(2j * math.pi * c_i * n / N)[:, None] * np.ones((1, 2))
        u_sub = dbp.subband_to_time(dbp.demux(np.fft.fft(tone, axis=0), n_sb), N)
        np.testing.assert_allclose(u_sub[i], 1.0, atol=1e-12)          # unit tone -> u_i == 1
        others = [l for l in range(n_sb) if l != i]
        if others:
            assert np.max(np.abs(u_sub[others])) < 1e-12
    u = _rand_field(N)
    u_sub = dbp.subband_to_time(dbp.demux(np.fft.fft(u, axis=0), n_sb), N)
    # Parseval: sum_i sum_k |u_i|^2 / R' = sum_n |u|^2 / R  with R' = R / N_sb
    assert np.sum(np.abs(u_sub) ** 2) * n_sb == pytest.approx(np.sum(np.abs(u) ** 2), rel=1e-12)
    # u[N_sb k] = sum_i exp(j 2 pi f_i k / R') u_i[k] with f_i / R' = c_i / N'
    k = np.arange(n_sub)
    rec = np.zeros((n_sub, 2), dtype=complex)
    for i in range(n_sb):
        c_i = -N // 2 + i * n_sub + n_sub // 2
        rec += np.exp(2j * math.pi * c_i * k / n_sub)[:, None] * u_sub[i]
    np.testing.assert_allclose(rec, u[::n_sb], atol=1e-12)
    # and back: time_to_subband inverts subband_to_time
    X = dbp.demux(np.fft.fft(u, axis=0), n_sb)
    np.testing.assert_allclose(dbp.time_to_subband(dbp.subband_to_time(X, N), N), X, atol=1e-9)


# ---------------------------------------------------------------------------------------------
def _closed_form_dispersion(u, beta2, Z, R):
    f = np.fft.fftfreq(u.shape[0], d=1.0 / R)
    w = 2 * math.pi * f
    return np.fft.ifft(np.fft.fft(u, axis=0) * np.exp(1j * beta2 * w ** 2 * Z / 2)[:, None], axis=0)


@pytest.mark.parametrize("n_sb,n_st,rho", [(1, 0, 0.5), (1, 1, 0.3), (2, 3, 0.12), (3, 2, 0.0),
                                           (5, 4, 1.0), (4, 15, 0.3)])
def test_linear_chain_equals_closed_form_dispersion(n_sb, n_st, rho):
    L = 480 * n_sb if n_sb != 4 else 1024
    R = 160e9
    beta2, Z = -21.7e-27, 240e3
    u = _rand_field(L)
    p = dbp.ChainParams(beta2=beta2, sample_rate=R, link_length=Z, n_sb=n_sb, ratio=rho,
                        taps=np.zeros((n_st, n_sb, n_sb, 5)))
    got = dbp.dbp_mode_u(u, p)
    want = _closed_form_dispersion(u, beta2, Z, R)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-11


def test_zero_dispersion_single_band_is_exact_spm_rotation():
    L, n_st = 256, 7
    u = _rand_field(L, scale=0.3)
    phi = RNG.uniform(0.05, 0.4, size=n_st)
    taps = signals.ssfm_delta_taps(n_st, 1, 9, phi)
    p = dbp.ChainParams(beta2=0.0, sample_rate=64e9, link_length=80e3, n_sb=1, ratio=0.3,
                        taps=taps)
    got = dbp.dbp_mode_u(u, p)
    I = np.abs(u[:, 0]) ** 2 + np.abs(u[:, 1]) ** 2
    want = u * np.exp(1j * np.sum(phi) * I)[:, None]
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_nlpr_preserves_energy_and_pointwise_intensity():
    N, n_sb = 5 * 64, 5
    u = _rand_field(N)
    taps = signals.random_taps(7, 3, n_sb, 11, 0.3, spread=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=320e9, link_length=240e3, n_sb=n_sb,
                        ratio=0.3, taps=taps)
    trace = []
    out = dbp.cbessfm_block(u, p, trace)
    pre = [a for n, a in trace if n == "pre_nlpr"]
    post = [a for n, a in trace if n == "post_nlpr"]
    assert len(pre) == len(post) == 3
    for a, b in zip(pre, post):
        Ia = np.abs(a[..., 0]) ** 2 + np.abs(a[..., 1]) ** 2
        Ib = np.abs(b[..., 0]) ** 2 + np.abs(b[..., 1]) ** 2
        np.testing.assert_allclose(Ib, Ia, rtol=1e-12)
    # total energy is preserved by every GVD and NLPR of the chain
    assert np.sum(np.abs(out) ** 2) == pytest.approx(np.sum(np.abs(u) ** 2), rel=1e-12)
    for a in pre:
        assert np.sum(np.abs(a) ** 2) * n_sb == pytest.approx(np.sum(np.abs(u) ** 2), rel=1e-12)


def test_time_domain_fir_equals_frequency_domain_mimo():
    # Fig. 3: the MIMO filter is done with RFFTs of the intensities and an N_sb x N_sb transfer
    # matrix obtained by FFT of the impulse responses (placed circularly at index m mod N').
    n_sb, n_sub, ntaps = 3, 64, 11
    P = RNG.uniform(0, 1, (n_sb, n_sub))
    w = RNG.standard_normal((n_sb, n_sb, ntaps))
    nc = ntaps // 2
    h = np.zeros((n_sb, n_sb, n_sub))
    for m in range(-nc, nc + 1):
        h[:, :, m % n_sub] = w[:, :, m + nc]
    H = np.fft.rfft(h, axis=2)
    Pf = np.fft.rfft(P, axis=1)
    theta_f = np.fft.irfft(np.einsum("ilk,lk->ik", H, Pf), n=n_sub, axis=1)
    np.testing.assert_allclose(dbp.nlpr_phase(P, w), theta_f, atol=1e-12)


def _textbook_asymmetric_ssfm(u, beta2, R, Z, n_st, rho, phi):
    """Plain lumped SSFM DBP: per step GVD((1-rho)dz), rotation exp(+j phi_s |u|^2), GVD(rho dz)."""
    f = np.fft.fftfreq(u.shape[0], d=1.0 / R)
    dz = Z / n_st
    H = lambda d: np.exp(1j * 2 * math.pi ** 2 * beta2 * d * f ** 2)[:, None]
    v = u.copy()
    for s in range(n_st):
        v = np.fft.ifft(np.fft.fft(v, axis=0) * H((1 - rho) * dz), axis=0)
        v = v * np.exp(1j * phi[s] * (np.abs(v[:, 0]) ** 2 + np.abs(v[:, 1]) ** 2))[:, None]
        v = np.fft.ifft(np.fft.fft(v, axis=0) * H(rho * dz), axis=0)
    return v


@pytest.mark.parametrize("rho", [0.5, 0.12, 0.0])
def test_single_band_delta_taps_equal_textbook_ssfm(rho):
    L, n_st = 1024, 6
    u = _rand_field(L, scale=0.4)
    phi = RNG.uniform(0.1, 0.3, n_st)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=64e9, link_length=480e3, n_sb=1,
                        ratio=rho, taps=signals.ssfm_delta_taps(n_st, 1, 5, phi))
    got = dbp.dbp_mode_u(u, p)
    want = _textbook_asymmetric_ssfm(u, -21.7e-27, 64e9, 480e3, n_st, rho, phi)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


def test_frequency_shift_equivariance_with_circulant_taps():
    # beta2 = 0 and taps that depend only on (l - i) mod N_sb: shifting the input spectrum by one
    # subband (a tone of frequency N' R / N) shifts every subband index by one.
    n_sb, n_sub, ntaps = 5, 32, 7
    N = n_sb * n_sub
    base = RNG.standard_normal((n_sb, ntaps)) * 0.2
    taps = np.zeros((2, n_sb, n_sb, ntaps))
    for i in range(n_sb):
        for l in range(n_sb):
            taps[:, i, l, :] = base[(l - i) % n_sb]
    p = dbp.ChainParams(beta2=0.0, sample_rate=160e9, link_length=160e3, n_sb=n_sb, ratio=0.3,
                        taps=taps)
    u = _rand_field(N, scale=0.5)
    shift = np.exp(2j * math.pi * n_sub * np.arange(N) / N)[:, None]
    a = dbp.cbessfm_block(u * shift, p)
    b = dbp.cbessfm_block(u, p) * shift
    np.testing.assert_allclose(a, b, atol=1e-12)
    # ... and the shift really matters for non-circulant taps (the check has teeth)
    taps2 = taps.copy()
    taps2[:, 0, 1, :] += 0.3
    p2 = dbp.ChainParams(beta2=0.0, sample_rate=160e9, link_length=160e3, n_sb=n_sb, ratio=0.3,
                         taps=taps2)
    assert np.max(np.abs(dbp.cbessfm_block(u * shift, p2) - dbp.cbessfm_block(u, p2) * shift)) > 1e-3


# ---------------------------------------------------------------------------------------------
def test_overlap_save_is_shift_equivariant_by_whole_blocks():
    n_sb, n_fft, ov = 2, 64, 16
    N, V = n_sb * n_fft, n_sb * (n_fft - ov)
    L = 7 * V
    u = _rand_field(L, scale=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=160e9, link_length=160e3, n_sb=n_sb,
                        ratio=0.3, taps=signals.random_taps(3, 2, n_sb, 5, 0.2))
    a = dbp.dbp_mode_b(np.roll(u, V, axis=0), p, n_fft, ov)
    b = np.roll(dbp.dbp_mode_b(u, p, n_fft, ov), V, axis=0)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_overlap_save_single_block_covering_sequence_equals_whole_sequence():
    n_sb, n_fft = 3, 64
    L = n_sb * n_fft
    u = _rand_field(L, scale=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=96e9, link_length=80e3, n_sb=n_sb,
                        ratio=0.3, taps=signals.random_taps(4, 2, n_sb, 5, 0.2))
    np.testing.assert_allclose(dbp.dbp_mode_b(u, p, n_fft, 0), dbp.dbp_mode_u(u, p), atol=1e-13)


def test_overlap_save_with_adequate_overlap_matches_whole_sequence():
    wl = configs.get_workload("c1_tiny")
    u, _ = signals.tx_waveform(wl, 0.0, seed=5)
    taps = signals.random_taps(11, 1, 1, 5, 0.02)
    p = dbp.ChainParams(beta2=wl.link.beta2, sample_rate=wl.signal.sample_rate,
                        link_length=wl.link.length, n_sb=1, ratio=0.5, taps=taps)
    whole = dbp.dbp_mode_u(u, p)
    # The truncation error of overlap-and-save falls as the overlap grows past the dispersion
    # memory (about 45 samples for 80 km at 64 GS/s); the slow decay is the Fresnel tail of the
    # band-limited dispersion kernel.
    errs = []
    for n_fft, ov in [(1024, 64), (1024, 128), (1024, 256), (2048, 1024)]:
        blk = dbp.dbp_mode_b(u, p, n_fft, ov)
        errs.append(np.linalg.norm(blk - whole) / np.linalg.norm(whole))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[2] < 2e-4 and errs[3] < 3e-5, errs
    blocks = dbp.dbp_mode_b(u, p, 1024, 256)
    # sampled evaluation of a subset of blocks gives the same samples
    part = dbp.dbp_mode_b(u, p, 1024, 256, blocks=[0, 5])
    V = 768
    np.testing.assert_array_equal(part[:V], blocks[:V])
    np.testing.assert_array_equal(part[5 * V: 6 * V], blocks[5 * V: 6 * V])
    assert np.isnan(part[V]).all()


@pytest.mark.parametrize("n_sb,n_st,rho", [(1, 2, 0.3), (3, 4, 0.12), (5, 3, 0.7)])
def test_reverse_chain_undoes_the_chain(n_sb, n_st, rho):
    """Applied in reverse, the steps of the chain are GVD(-rho L), rotation by exp(-j theta_N),
    GVD(-L), ..., rotation by exp(-j theta_1), GVD(-(1 - rho) L).  That is the chain itself
    with -beta2, ratio 1 - rho and taps -w[N_st - 1 - s], so running it on the output must give
    the input back; the rotation phase is recomputed from the rotated field's own intensity."""
    L = 96 * n_sb
    u = _rand_field(L, scale=0.5)
    taps = signals.random_taps(7, n_st, n_sb, 7, 0.8, spread=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=64e9 * n_sb, link_length=320e3, n_sb=n_sb,
                        ratio=rho, taps=taps)
    inv = dbp.ChainParams(beta2=21.7e-27, sample_rate=64e9 * n_sb, link_length=320e3,
                          n_sb=n_sb, ratio=1.0 - rho, taps=-taps[::-1].copy())
    out = dbp.dbp_mode_u(u, p)
    assert np.linalg.norm(out - u) > 0.1 * np.linalg.norm(u)        # the chain did something
    back = dbp.dbp_mode_u(out, inv)
    assert np.linalg.norm(back - u) / np.linalg.norm(u) < 1e-12
