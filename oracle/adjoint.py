"""Reverse-mode gradient of the CB-ESSFM chain in FP64 -- oracle (test infrastructure only).

The paper optimizes the taps offline with finite-difference gradients (Sec. III-B) and names
automatic differentiation as the natural next step; this module is the exact adjoint of
``oracle.dbp`` used to check the GPU adjoint kernel.

Gradient convention: for a real loss and a complex variable z, ``G_z = dL/dRe(z) + j dL/dIm(z)``
(what a real-view autograd returns), so ``dL = Re(sum conj(G_z) dz)``.  A complex-linear map
y = A x then back-propagates as G_x = A^H G_y.  Through the rotation v' = v exp(j theta) of
Fig. 3:  G_theta = -Im(sum_pol conj(G_v') v'),  G_v = exp(-j theta) G_v' + 2 G_P v,  with the FIR
and intensity terms  G_w[i,l,m] = sum_k G_theta_i[k] P_l[(k - m) mod N'],
G_P_l[n] = sum_i sum_m w[i,l,m] G_theta_i[(n + m) mod N'].  The splitting ratio enters only the
first and last GVD (Sec. III-C): dh_first/drho = -j 2 pi^2 beta2 L_step f^2 h_first and
dh_last/drho = +j 2 pi^2 beta2 L_step f^2 h_last.

Per-polarization NLPR (Eqs. (NLPR_polx), (NLPR_poly)): each polarization p has its own phase,
theta^p_i = sum_l sum_m [a^p_il[m] Px_l + b^p_il[m] Py_l][k - m], with a = b = w_ii on the
diagonal and, for l != i, (a^x, b^x) = (2, 1) w_il / 1.5 and (a^y, b^y) = (1, 2) w_il / 1.5.  Then
G_theta^p = -Im(conj(G_v'^p) v'^p) per polarization, G_Px_l[n] = sum_i sum_m (a^x_il[m]
G_theta^x_i + a^y_il[m] G_theta^y_i)[n + m] (and G_Py with b), G_v^p = exp(-j theta^p) G_v'^p +
2 G_Pp v^p, and G_w_il[m] = sum_k G_theta^x_i[k] (a^x Px + b^x Py)_l[k - m] / w + the same for y
(the coefficients are linear in w).
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np

from .dbp import (ChainParams, subband_bins, demux, mux, gvd_factor, subband_to_time,
                  time_to_subband, nlpr_phase, nlpr_phase_per_pol, ols_geometry,
                  ols_block_input)


def _fir_adjoint(G_theta: np.ndarray, P: np.ndarray, w: np.ndarray):
    """Adjoint of theta = FIR(P; w): returns (G_P, G_w)."""
    n_sb, n_sub = P.shape
    ntaps = w.shape[2]
    nc = ntaps // 2
    G_P = np.zeros_like(P)
    G_w = np.zeros_like(w)
    for i in range(n_sb):
        for l in range(n_sb):
            for m in range(-nc, nc + 1):
                G_w[i, l, m + nc] = np.sum(G_theta[i] * np.roll(P[l], m))
                # theta_i[k] gets w P_l[k - m]  ->  P_l[n] feeds theta_i[n + m]
                G_P[l] += w[i, l, m + nc] * np.roll(G_theta[i], -m)
    return G_P, G_w


def _per_pol_weights(i: int, l: int):
    """(a^x, b^x, a^y, b^y) of the per-polarization phase per unit effective tap w_il."""
    if i == l:
        return 1.0, 1.0, 1.0, 1.0
    return 2.0 / 1.5, 1.0 / 1.5, 1.0 / 1.5, 2.0 / 1.5


def _fir_adjoint_per_pol(G_tx: np.ndarray, G_ty: np.ndarray, Px: np.ndarray, Py: np.ndarray,
                         w: np.ndarray):
    """Adjoint of (theta^x, theta^y) = nlpr_phase_per_pol(Px, Py; w): (G_Px, G_Py, G_w)."""
    n_sb, n_sub = Px.shape
    ntaps = w.shape[2]
    nc = ntaps // 2
    G_Px, G_Py = np.zeros_like(Px), np.zeros_like(Py)
    G_w = np.zeros_like(w)
    for i in range(n_sb):
        for l in range(n_sb):
            ax, bx, ay, by = _per_pol_weights(i, l)
            for m in range(-nc, nc + 1):
                px, py = np.roll(Px[l], m), np.roll(Py[l], m)
                G_w[i, l, m + nc] = (np.sum(G_tx[i] * (ax * px + bx * py))
                                     + np.sum(G_ty[i] * (ay * px + by * py)))
                gx, gy = np.roll(G_tx[i], -m), np.roll(G_ty[i], -m)
                G_Px[l] += w[i, l, m + nc] * (ax * gx + ay * gy)
                G_Py[l] += w[i, l, m + nc] * (bx * gx + by * gy)
    return G_Px, G_Py, G_w


def cbessfm_block_vjp(u: np.ndarray, p: ChainParams, G_out: np.ndarray
                      ) -> Tuple[np.ndarray, np.ndarray, float]:
    """Vector-Jacobian product of ``oracle.dbp.cbessfm_block`` on one block.

    Returns (G_in (N, 2) complex, G_taps like p.taps, G_ratio float).
    """
    N = u.shape[0]
    n_sb = p.n_sb
    _, b = subband_bins(N, n_sb)
    freq = b * (p.sample_rate / N)
    Ls = p.step_length
    kdisp = 2.0 * math.pi ** 2 * p.beta2 * Ls * freq ** 2        # d(phase)/d(length share)

    # ---- forward, keeping what the backward pass needs -------------------------------------
    X0 = demux(np.fft.fft(u, axis=0), n_sb)
    G_taps = np.zeros_like(p.taps)
    if p.n_st == 0:
        h_all = gvd_factor(p.beta2, p.link_length, freq)[..., None]
        G_X = demux(np.fft.fft(G_out, axis=0), n_sb) / N           # adjoint of ifft, mux
        G_X0 = np.conj(h_all) * G_X
        G_in = N * np.fft.ifft(mux(G_X0), axis=0)
        return G_in, G_taps, 0.0
    h_first = gvd_factor(p.beta2, (1.0 - p.ratio) * Ls, freq)[..., None]
    h_int = gvd_factor(p.beta2, Ls, freq)[..., None]
    h_last = gvd_factor(p.beta2, p.ratio * Ls, freq)[..., None]
    X = X0 * h_first
    saved = []
    for s in range(p.n_st):
        v = subband_to_time(X, N)
        if p.per_pol:
            P = (np.abs(v[..., 0]) ** 2, np.abs(v[..., 1]) ** 2)
            theta = np.stack(nlpr_phase_per_pol(P[0], P[1], p.taps[s]), axis=-1)  # (.., pol)
        else:
            P = np.abs(v[..., 0]) ** 2 + np.abs(v[..., 1]) ** 2
            theta = nlpr_phase(P, p.taps[s])[..., None]
        vr = v * np.exp(1j * theta)
        saved.append((v, P, theta, vr))
        X = time_to_subband(vr, N)
        X = X * (h_int if s < p.n_st - 1 else h_last)
    X_before_last = X / h_last                                    # spectrum entering the last GVD

    # ---- backward ---------------------------------------------------------------------------
    G_X = demux(np.fft.fft(G_out, axis=0), n_sb) / N               # (ifft)^H = fft / N ; mux^H
    G_ratio = float(np.sum(np.real(np.conj(G_X) * (1j * kdisp[..., None]) * h_last
                                   * X_before_last)))
    for s in range(p.n_st - 1, -1, -1):
        h = h_int if s < p.n_st - 1 else h_last
        G_X = np.conj(h) * G_X
        # X = (N/N') F v'  ->  G_v' = (N/N') F^H G_X = N ifft(G_X)
        G_vr = N * np.fft.ifft(G_X, axis=1)
        v, P, theta, vr = saved[s]
        if p.per_pol:
            G_tp = -np.imag(np.conj(G_vr) * vr)                    # per polarization
            G_Px, G_Py, G_w = _fir_adjoint_per_pol(G_tp[..., 0], G_tp[..., 1], P[0], P[1],
                                                   p.taps[s])
            G_P = np.stack([G_Px, G_Py], axis=-1)
        else:
            G_theta = -np.imag(np.sum(np.conj(G_vr) * vr, axis=-1))
            G_Pm, G_w = _fir_adjoint(G_theta, P, p.taps[s])
            G_P = G_Pm[..., None]
        G_taps[s] = G_w
        G_v = np.exp(-1j * theta) * G_vr + 2.0 * G_P * v
        # v = (1/N) F^H X  ->  G_X = (1/N) F G_v
        G_X = np.fft.fft(G_v, axis=1) / N
    G_ratio += float(np.sum(np.real(np.conj(G_X) * (-1j * kdisp[..., None]) * h_first * X0)))
    G_X0 = np.conj(h_first) * G_X
    G_in = N * np.fft.ifft(mux(G_X0), axis=0)                      # U0 = F u -> G_u = F^H G_U0
    return G_in, G_taps, G_ratio


def dbp_mode_b_vjp(field: np.ndarray, p: ChainParams, n_fft: int, overlap: int,
                   G_out: np.ndarray) -> Tuple[np.ndarray, np.ndarray, float]:
    """VJP of ``oracle.dbp.dbp_mode_b``: only the kept samples of each block carry gradient."""
    field = np.asarray(field, dtype=np.complex128)
    L = field.shape[0]
    N = p.n_sb * n_fft
    n_ov = p.n_sb * overlap
    V, n_blocks = ols_geometry(L, N, n_ov)
    G_in = np.zeros((L, 2), dtype=np.complex128)
    G_taps = np.zeros_like(p.taps)
    G_ratio = 0.0
    for b in range(n_blocks):
        n_keep = min(V, L - b * V)
        Gb = np.zeros((N, 2), dtype=np.complex128)
        Gb[n_ov // 2: n_ov // 2 + n_keep] = G_out[b * V: b * V + n_keep]
        gi, gt, gr = cbessfm_block_vjp(ols_block_input(field, b, N, n_ov), p, Gb)
        idx = np.mod(b * V - n_ov // 2 + np.arange(N), L)
        np.add.at(G_in, idx, gi)
        G_taps += gt
        G_ratio += gr
    return G_in, G_taps, G_ratio
