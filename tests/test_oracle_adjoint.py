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
