"""Analytic CB-ESSFM coefficients in FP64 -- oracle (test infrastructure only).

Sec. II-D of the paper.  The NLPR of subband i driven by the intensity of subband l has the
impulse response

    c_il[m] = (P / R'^2) double-integral over mu, nu in [f_il - R'/2, f_il + R'/2] of
              K(mu, nu) exp(j 2 pi (mu - nu) m / R')                  (Eq. ESSFM_coefficients_general)

with f_il = f_l - f_i and the frequency-domain Volterra kernel of one step of length L

    K(mu, nu) = integral_{-L/2}^{L/2} gamma g(z) H(z, mu) H*(z, nu) H(-z, mu - nu) dz
              = integral gamma g(z) exp(-j 2 b z) dz,   b = 2 pi^2 beta2 nu (mu - nu)
                                                                  (Eqs. kernel_definition, kernel_b)

where H(z, f) = exp(-j 2 pi^2 beta2 f^2 z) and g(z) is the normalized power profile: N_sp
identical spans of length L / N_sp, each starting at unit power and decaying as exp(-alpha zeta).
For that profile the paper gives the closed form (Eq. kernel_analytic)

    K = gamma exp(-a L_sp) sinh((a + j b) L_sp) sin(b L) / ((a + j b) sin(b L_sp)),  a = alpha/2.

The double integral is evaluated as the paper suggests, from the kernel on a square grid of
frequencies: an M x M midpoint rule, whose diagonal sums are a two-dimensional DFT of the grid.

Readings taken here (where the paper is silent or ambiguous):
* The spans of a step start at z = -L/2 + n L_sp (the appendix places them at multiples of L_sp
  for even N_sp, which is the same grid).
* K(mu, nu) is not Hermitian (K(mu, nu) != conj K(nu, mu)), so c_il[m] is complex in general;
  the NLPR is a real phase, so the taps are the real parts.  Only the SPM response of a lossless
  step is real.
* The DBP taps of step s are w[s][i][l][m + N_c] = Re c_il[m] for l = i and (3/2) Re c_il[m]
  for l != i (Eq. NLPR-multiband-2pol), with P the power at the input of the step.
"""
from __future__ import annotations

import math

import numpy as np


def kernel_closed_form(mu, nu, beta2: float, gamma: float, alpha: float, step_length: float,
                       n_spans: int = 1):
    """K(mu, nu) of Eq. (kernel_analytic), with its limits at b -> 0 and a + j b -> 0."""
    mu = np.asarray(mu, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    L = float(step_length)
    Lsp = L / n_spans
    a = alpha / 2.0
    b = 2.0 * math.pi ** 2 * beta2 * nu * (mu - nu)
    x = (a + 1j * b) * Lsp
    small = np.abs(x) < 1e-8
    xs = np.where(small, 1.0, x)
    sinhc = np.where(small, 1.0 + x * x / 6.0, np.sinh(xs) / xs)          # sinh(x) / x
    s_step = np.sin(b * L)
    s_span = np.sin(b * Lsp)
    # sin(N y) / sin(y) -> N (-1)^{k (N - 1)} where y = k pi
    k = np.round(b * Lsp / math.pi)
    limit = n_spans * np.where((k * (n_spans - 1)) % 2 == 0, 1.0, -1.0)
    near = np.abs(s_span) < 1e-12
    ratio = np.where(near, limit, s_step / np.where(near, 1.0, s_span))
    return gamma * math.exp(-a * Lsp) * Lsp * sinhc * ratio


def kernel_numeric(mu, nu, beta2: float, gamma: float, alpha: float, step_length: float,
                   n_spans: int = 1, nodes: int = 64):
    """K(mu, nu) of Eq. (kernel_definition) by Gauss-Legendre quadrature over each span."""
    mu = np.asarray(mu, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    L = float(step_length)
    Lsp = L / n_spans
    t, wts = np.polynomial.legendre.leggauss(nodes)
    b = 2.0 * math.pi ** 2 * beta2 * nu * (mu - nu)
    total = np.zeros(np.broadcast(mu, nu).shape, dtype=np.complex128)
    for n in range(n_spans):
        z0 = -L / 2.0 + n * Lsp
        zeta = 0.5 * Lsp * (t + 1.0)                                     # position in the span
        z = z0 + zeta
        for zz, ze, w in zip(z, zeta, wts):
            # H(z, mu) H*(z, nu) H(-z, mu - nu), H(z, f) = exp(-j 2 pi^2 beta2 f^2 z)
            h = (np.exp(-1j * 2 * math.pi ** 2 * beta2 * mu ** 2 * zz)
                 * np.conj(np.exp(-1j * 2 * math.pi ** 2 * beta2 * nu ** 2 * zz))
                 * np.exp(-1j * 2 * math.pi ** 2 * beta2 * (mu - nu) ** 2 * (-zz)))
            total += gamma * math.exp(-alpha * ze) * h * (0.5 * Lsp * w)
    return total


def coefficients(beta2: float, gamma: float, alpha: float, step_length: float, n_spans: int,
                 power: float, rate_sub: float, f_sep: float, ntaps: int, grid: int):
    """Complex c[m], m = -N_c .. N_c, of Eq. (ESSFM_coefficients_general) on a grid x grid
    midpoint rule over [f_sep - R'/2, f_sep + R'/2]^2 (rate_sub = R')."""
    nc = (ntaps - 1) // 2
    M = int(grid)
    f = f_sep - rate_sub / 2.0 + (np.arange(M) + 0.5) * rate_sub / M
    K = kernel_closed_form(f[:, None], f[None, :], beta2, gamma, alpha, step_length, n_spans)
    p = np.arange(M)
    out = np.zeros(2 * nc + 1, dtype=np.complex128)
    for idx, m in enumerate(range(-nc, nc + 1)):
        # (mu_p - nu_q) / R' = (p - q) / M
        e = np.exp(1j * 2 * math.pi * np.subtract.outer(p, p) * m / M)
        out[idx] = power / M ** 2 * np.sum(K * e)
    return out


def dbp_taps(beta2: float, gamma: float, alpha: float, step_length: float, n_spans: int,
             step_powers, sample_rate: float, n_sb: int, ntaps: int, grid: int) -> np.ndarray:
    """Effective DBP taps [n_st][n_sb][n_sb][ntaps]: Re c_il[m] with the 3/2 XPM factor folded
    in, subband spacing R' = R / N_sb, P = step_powers[s] for step s."""
    step_powers = np.asarray(step_powers, dtype=np.float64)
    n_st = step_powers.shape[0]
    rate_sub = sample_rate / n_sb
    out = np.zeros((n_st, n_sb, n_sb, ntaps), dtype=np.float64)
    for s in range(n_st):
        for i in range(n_sb):
            for l in range(n_sb):
                c = coefficients(beta2, gamma, alpha, step_length, n_spans, step_powers[s],
                                 rate_sub, (l - i) * rate_sub, ntaps, grid)
                out[s, i, l] = np.real(c) * (1.0 if i == l else 1.5)
    return out
