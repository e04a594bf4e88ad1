"""Pins of the FP64 adjoint (oracle.adjoint) against central finite differences of the forward
oracle and the dot-product identity <G_out, J v> = Re<J^T G_out, v>, for the Manakov NLPR and the
per-polarization NLPR of Eqs. (NLPR_polx), (NLPR_poly).
"""
import math

import numpy as np
import pytest

from oracle import adjoint, dbp
from synth import signals


def _setup(n_sb=3, n_fft=32, ov=8, n_st=2, ntaps=5, L=None, seed=0, per_pol=False):
    rng = np.random.default_rng(seed)
    L = L or 4 * n_sb * (n_fft - ov) + 7 * n_sb
    u = 0.6 * (rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2)))
    taps = signals.random_taps(seed + 1, n_st, n_sb, ntaps, 0.3, spread=0.5)
    p = dbp.ChainParams(beta2=-21.7e-27, sample_rate=96e9 * n_sb / 3, link_length=160e3,
                        n_sb=n_sb, ratio=0.3, taps=taps, per_pol=per_pol)
    target = 0.6 * (rng.standard_normal((L, 2)) + 1j * rng.standard_normal((L, 2)))
    return u, p, target, n_fft, ov


def _loss(u, p, n_fft, ov, target):
    out = dbp.dbp_mode_b(u, p, n_fft, ov)
    return float(np.sum(np.abs(out - target) ** 2)), out


def _with(p, taps=None, ratio=None):
    return dbp.ChainParams(p.beta2, p.sample_rate, p.link_length, p.n_sb,
                           p.ratio if ratio is None else ratio,
                           p.taps if taps is None else taps, per_pol=p.per_pol)


@pytest.mark.parametrize("n_sb,n_st,per_pol", [(1, 1, False), (3, 2, False), (2, 3, False),
                                               (3, 2, True), (2, 3, True), (1, 2, True)])
def test_tap_and_ratio_gradients_match_central_differences(n_sb, n_st, per_pol):
    u, p, target, n_fft, ov = _setup(n_sb=n_sb, n_st=n_st, per_pol=per_pol)
    f0, out = _loss(u, p, n_fft, ov, target)
    G_out = 2.0 * (out - target)                  # dL/dRe + j dL/dIm of sum |out - t|^2
    _, G_taps, G_ratio = adjoint.dbp_mode_b_vjp(u, p, n_fft, ov, G_out)
    h = 1e-6
    rng = np.random.default_rng(5)
    idx = [tuple(rng.integers(0, s) for s in p.taps.shape) for _ in range(6)]
    for ix in idx:
        tp, tm = p.taps.copy(), p.taps.copy()
        tp[ix] += h
        tm[ix] -= h
        fp, _ = _loss(u, _with(p, taps=tp), n_fft, ov, target)
        fm, _ = _loss(u, _with(p, taps=tm), n_fft, ov, target)
        fd = (fp - fm) / (2 * h)
        assert G_taps[ix] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(f0)), ix
    fp, _ = _loss(u, _with(p, ratio=p.ratio + h), n_fft, ov, target)
    fm, _ = _loss(u, _with(p, ratio=p.ratio - h), n_fft, ov, target)
    assert G_ratio == pytest.approx((fp - fm) / (2 * h), rel=1e-6)


def test_per_pol_diagonal_and_coupling_taps_both_checked():
    """The per-polarization weights differ between the self-band (l = i) and the coupling
    (l != i) taps: check one of each against central differences."""
    u, p, target, n_fft, ov = _setup(n_sb=2, n_st=1, per_pol=True, seed=3)
    f0, out = _loss(u, p, n_fft, ov, target)
    _, G_taps, _ = adjoint.dbp_mode_b_vjp(u, p, n_fft, ov, 2.0 * (out - target))
    h = 1e-6
    for ix in [(0, 0, 0, 2), (0, 1, 0, 1), (0, 0, 1, 3), (0, 1, 1, 2)]:
        tp, tm = p.taps.copy(), p.taps.copy()
        tp[ix] += h
        tm[ix] -= h
        fd = (_loss(u, _with(p, taps=tp), n_fft, ov, target)[0]
              - _loss(u, _with(p, taps=tm), n_fft, ov, target)[0]) / (2 * h)
        assert G_taps[ix] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(f0)), ix


@pytest.mark.parametrize("per_pol", [False, True])
def test_input_gradient_dot_product_identity(per_pol):
    u, p, target, n_fft, ov = _setup(n_sb=2, n_st=2, per_pol=per_pol)
    rng = np.random.default_rng(8)
    G_out = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    v = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    G_in, _, _ = adjoint.dbp_mode_b_vjp(u, p, n_fft, ov, G_out)
    eps = 1e-6
    Jv = (dbp.dbp_mode_b(u + eps * v, p, n_fft, ov) -
          dbp.dbp_mode_b(u - eps * v, p, n_fft, ov)) / (2 * eps)
    lhs = np.sum(np.real(np.conj(G_out) * Jv))
    rhs = np.sum(np.real(np.conj(G_in) * v))
    assert lhs == pytest.approx(rhs, rel=1e-7)


def test_zero_steps_adjoint_is_conjugate_dispersion():
    u, p, target, n_fft, ov = _setup(n_sb=2, n_st=2)
    p0 = dbp.ChainParams(p.beta2, p.sample_rate, p.link_length, p.n_sb, p.ratio,
                         np.zeros((0, 2, 2, 5)))
    rng = np.random.default_rng(3)
    N = p.n_sb * n_fft
    G = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    x = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    G_in, _, gr = adjoint.cbessfm_block_vjp(x, p0, G)
    # the chain is unitary and linear: its adjoint is its inverse, i.e. dispersion of -Z
    pinv = dbp.ChainParams(p.beta2, p.sample_rate, -p.link_length, p.n_sb, p.ratio,
                           np.zeros((0, 2, 2, 5)))
    np.testing.assert_allclose(G_in, dbp.cbessfm_block(G, pinv), atol=1e-12)
    assert gr == 0.0


def test_per_pol_fir_adjoint_equals_its_sum_difference_form():
    """The adjoint of the per-polarization FIR (weights (1, 1) on the own band, (2, 1)/1.5 and
    (1, 2)/1.5 on the others, Eqs. (NLPR_polx), (NLPR_poly)) rewritten with S = G_tx + G_ty and
    D = G_tx - G_ty: G_Px/y,l = sum_i corr(w_il, S_i) +/- (1/3) sum_{i != l} corr(w_il, D_i),
    dL/dw_il[m] = sum_k S_i[k] (Px + Py)_l[k - m] + [i != l] (1/3) sum_k D_i[k] (Px - Py)_l[k - m]."""
    from oracle import adjoint as oa
    rng = np.random.default_rng(21)
    n_sb, n, ntaps = 3, 32, 5
    nc = ntaps // 2
    Px, Py = rng.random((n_sb, n)), rng.random((n_sb, n))
    G_tx, G_ty = rng.standard_normal((n_sb, n)), rng.standard_normal((n_sb, n))
    w = rng.standard_normal((n_sb, n_sb, ntaps))
    G_Px, G_Py, G_w = oa._fir_adjoint_per_pol(G_tx, G_ty, Px, Py, w)
    S, D = G_tx + G_ty, G_tx - G_ty
    want_x, want_y, want_w = np.zeros_like(Px), np.zeros_like(Py), np.zeros_like(w)
    for i in range(n_sb):
        for l in range(n_sb):
            cross = 1.0 / 3.0 if i != l else 0.0
            for m in range(-nc, nc + 1):
                s_term = w[i, l, m + nc] * np.roll(S[i], -m)
                d_term = cross * w[i, l, m + nc] * np.roll(D[i], -m)
                want_x[l] += s_term + d_term
                want_y[l] += s_term - d_term
                want_w[i, l, m + nc] = (np.sum(S[i] * np.roll(Px[l] + Py[l], m))
                                        + cross * np.sum(D[i] * np.roll(Px[l] - Py[l], m)))
    np.testing.assert_allclose(G_Px, want_x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(G_Py, want_y, rtol=0, atol=1e-12)
    np.testing.assert_allclose(G_w, want_w, rtol=0, atol=1e-12)
