"""CB-ESSFM digital backpropagation in FP64 -- oracle (test infrastructure only).

Follows the paper's Sec. III-A (Figs. 2-3): per block of N 4D samples, two full-band CFFTs, a
DEMUX into N_sb subbands of N' = N / N_sb bins, then N_st times {GVD, NLPR} with the NLPR of
Eq. (NLPR-multiband-2pol) done in the time domain of each subband, a final GVD, MUX and two
inverse CFFTs of size N.  The GVD of a frequency component f over a length dz is
h = exp(+j 2 pi^2 beta2 dz f^2) (Sec. III-A, the inverse of Eq. (GVD_transfer-function)).  With
asymmetric steps (Sec. III-C) the first GVD covers (1 - rho) L_step, the interior ones L_step and
the last one rho L_step.

Readings of the paper taken here (where it is silent or ambiguous):
* Subband i (0-based) owns the centred bins b in [-N/2 + i N', -N/2 + (i+1) N'); its centre is
  c_i = -N/2 + i N' + N'/2 and its lowpass samples are
  u_i[k] = (1/N) sum_{k'} X[c_i + k'] exp(+j 2 pi k' k / N'), k' in [-N'/2, N'/2), so a unit tone
  at f_i gives u_i = 1 and the subbands sum back to u (Eq. (subband-division)).
* Each subband bin keeps its absolute frequency f = (c_i + k') R / N in the GVD (walk-off kept).
* The NLPR uses the [k - m] index of Eq. (NLPR-multiband-2pol), circular in the block:
  theta_i[k] = sum_l sum_{m=-Nc}^{Nc} w[i][l][m + Nc] P_l[(k - m) mod N'] with
  P_l = |x_l|^2 + |y_l|^2; the taps are the effective ones (3/2 XPM factor folded in).
* DBP rotates by exp(+j theta) (the forward model rotates by exp(-j theta), Eq. (ESSFM-model_b),
  and DBP reverses the sign of the parameters).
* The input is one period of a periodic sequence: overlap-and-save blocks wrap circularly.
* With N_st = 0 the chain is a single GVD over the whole link (EDC).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np


@dataclass
class ChainParams:
    beta2: float            # s^2/m of the fiber being backpropagated
    sample_rate: float      # full-band rate R (Hz)
    link_length: float      # m; the step length is link_length / n_st
    n_sb: int               # subbands N_sb
    ratio: float            # splitting ratio rho
    taps: np.ndarray        # (n_st, n_sb, n_sb, ntaps) effective taps, float64
    per_pol: bool = False   # full-complexity NLPR of Eqs. (NLPR_polx), (NLPR_poly)

    @property
    def n_st(self) -> int:
        return int(self.taps.shape[0])

    @property
    def ntaps(self) -> int:
        return int(self.taps.shape[3])

    @property
    def step_length(self) -> float:
        return self.link_length / self.n_st if self.n_st > 0 else 0.0


# ---------------------------------------------------------------------------------------------
# Subband bookkeeping (Sec. III-A: DEMUX "at no cost in the frequency domain")
# ---------------------------------------------------------------------------------------------

def subband_bins(n_block: int, n_sb: int):
    """For every subband i and DFT index kappa in [0, N'): (full-band DFT index, centred bin).

    Returns two int arrays of shape (n_sb, N'): ``K`` (index into the length-N DFT) and ``b``
    (centred bin number in [-N/2, N/2), frequency b R / N).
    """
    assert n_block % n_sb == 0
    n_sub = n_block // n_sb
    assert n_sub % 2 == 0 and n_block % 2 == 0, "even block and subband sizes"
    kappa = np.arange(n_sub)
    k_rel = np.where(kappa < n_sub // 2, kappa, kappa - n_sub)        # k' in [-N'/2, N'/2)
    b = np.empty((n_sb, n_sub), dtype=np.int64)
    for i in range(n_sb):
        c_i = -n_block // 2 + i * n_sub + n_sub // 2
        b[i] = c_i + k_rel
    K = np.mod(b, n_block)
    return K, b


def demux(U: np.ndarray, n_sb: int) -> np.ndarray:
    """Full-band spectrum (N, 2) -> subband spectra (n_sb, N', 2); bins keep their values."""
    K, _ = subband_bins(U.shape[0], n_sb)
    return U[K, :].copy()


def mux(X: np.ndarray) -> np.ndarray:
    """Inverse of ``demux``: subband spectra (n_sb, N', 2) -> full-band spectrum (N, 2)."""
    n_sb, n_sub, _ = X.shape
    K, _ = subband_bins(n_sb * n_sub, n_sb)
    U = np.zeros((n_sb * n_sub, 2), dtype=np.complex128)
    U[K.reshape(-1), :] = X.reshape(-1, 2)
    return U


def gvd_factor(beta2: float, dz: float, freq: np.ndarray) -> np.ndarray:
    """GVD compensation h = exp(+j 2 pi^2 beta2 dz f^2) (Sec. III-A)."""
    return np.exp(1j * 2.0 * math.pi ** 2 * beta2 * dz * freq ** 2)


def subband_to_time(X: np.ndarray, n_block: int) -> np.ndarray:
    """u_i[k] = (1/N) sum_k' X_i[k'] exp(+j 2 pi k' k / N')  (per subband and polarization)."""
    n_sub = X.shape[1]
    return np.fft.ifft(X, axis=1) * (n_sub / n_block)


def time_to_subband(u: np.ndarray, n_block: int) -> np.ndarray:
    """Inverse of ``subband_to_time``: X_i = (N / N') DFT_{N'}(u_i) = N_sb DFT_{N'}(u_i)."""
    n_sub = u.shape[1]
    return np.fft.fft(u, axis=1) * (n_block / n_sub)


def nlpr_phase(P: np.ndarray, w: np.ndarray) -> np.ndarray:
    """theta_i[k] = sum_l sum_{m=-Nc}^{Nc} w[i, l, m + Nc] P_l[(k - m) mod N'].

    Eq. (NLPR-multiband-2pol) with effective taps, evaluated as a circular time-domain sum.
    P: (n_sb, N') real intensities; w: (n_sb, n_sb, ntaps).
    """
    n_sb, n_sub = P.shape
    ntaps = w.shape[2]
    nc = ntaps // 2
    theta = np.zeros((n_sb, n_sub), dtype=np.float64)
    for i in range(n_sb):
        for l in range(n_sb):
            for m in range(-nc, nc + 1):
                # np.roll(a, m)[k] = a[(k - m) mod N']
                theta[i] += w[i, l, m + nc] * np.roll(P[l], m)
    return theta


def nlpr_phase_per_pol(Px: np.ndarray, Py: np.ndarray, w: np.ndarray):
    """(theta^x, theta^y) of Eqs. (NLPR_polx), (NLPR_poly), circular in the block.

    theta^x_i[k] = sum_m c_ii[m] (Px_i + Py_i)[k - m] + sum_{l != i} sum_m c_il[m] (2 Px_l + Py_l)[k - m]
    and theta^y_i with (Px_l + 2 Py_l).  The taps w are the effective ones of the Manakov form
    (w_ii = c_ii, w_il = (3/2) c_il), so c_il = w_il / 1.5 here; the index is [k - m] as in the
    Manakov form.  With Px = Py both reduce to Eq. (NLPR-multiband-2pol).
    """
    n_sb, n_sub = Px.shape
    ntaps = w.shape[2]
    nc = ntaps // 2
    tx = np.zeros((n_sb, n_sub), dtype=np.float64)
    ty = np.zeros((n_sb, n_sub), dtype=np.float64)
    for i in range(n_sb):
        for l in range(n_sb):
            for m in range(-nc, nc + 1):
                px, py = np.roll(Px[l], m), np.roll(Py[l], m)
                if l == i:
                    c = w[i, l, m + nc]
                    tx[i] += c * (px + py)
                    ty[i] += c * (px + py)
                else:
                    c = w[i, l, m + nc] / 1.5
                    tx[i] += c * (2.0 * px + py)
                    ty[i] += c * (px + 2.0 * py)
    return tx, ty


def nlpr(u: np.ndarray, w: np.ndarray, per_pol: bool = False) -> np.ndarray:
    """Nonlinear phase rotation of all subbands (Fig. 3): intensity, MIMO FIR, rotation.

    u: (n_sb, N', 2) subband time samples (x, y); returns u * exp(+j theta_i) on both pols, or
    x * exp(+j theta^x_i), y * exp(+j theta^y_i) with ``per_pol``.
    """
    if per_pol:
        Px, Py = np.abs(u[..., 0]) ** 2, np.abs(u[..., 1]) ** 2
        tx, ty = nlpr_phase_per_pol(Px, Py, w)
        return np.stack([u[..., 0] * np.exp(1j * tx), u[..., 1] * np.exp(1j * ty)], axis=-1)
    P = np.abs(u[..., 0]) ** 2 + np.abs(u[..., 1]) ** 2
    theta = nlpr_phase(P, w)
    return u * np.exp(1j * theta)[..., None]


def cbessfm_block(u: np.ndarray, p: ChainParams, trace: Optional[List] = None) -> np.ndarray:
    """The CB-ESSFM chain on one circular block u of shape (N, 2) (Fig. 3).

    If ``trace`` is a list, (stage name, array copy) pairs are appended for tests.
    """
    N = u.shape[0]
    n_sb = p.n_sb
    _, b = subband_bins(N, n_sb)
    freq = b * (p.sample_rate / N)
    U = np.fft.fft(u, axis=0)                          # two full-band CFFTs (x and y)
    X = demux(U, n_sb)
    if trace is not None:
        trace.append(("demux", X.copy()))
    if p.n_st == 0:
        X = X * gvd_factor(p.beta2, p.link_length, freq)[..., None]
    else:
        Ls = p.step_length
        X = X * gvd_factor(p.beta2, (1.0 - p.ratio) * Ls, freq)[..., None]
        for s in range(p.n_st):
            us = subband_to_time(X, N)
            if trace is not None:
                trace.append(("pre_nlpr", us.copy()))
            us = nlpr(us, p.taps[s], p.per_pol)
            if trace is not None:
                trace.append(("post_nlpr", us.copy()))
            X = time_to_subband(us, N)
            dz = Ls if s < p.n_st - 1 else p.ratio * Ls
            X = X * gvd_factor(p.beta2, dz, freq)[..., None]
    U = mux(X)
    return np.fft.ifft(U, axis=0)                      # two inverse CFFTs of size N


# ---------------------------------------------------------------------------------------------
# Whole-sequence forms
# ---------------------------------------------------------------------------------------------

def dbp_mode_u(field: np.ndarray, p: ChainParams) -> np.ndarray:
    """Mode U: the chain on the whole (periodic) sequence as one block."""
    return cbessfm_block(np.asarray(field, dtype=np.complex128), p)


def ols_geometry(L: int, n_block: int, n_ov: int):
    """Overlap-and-save geometry (Sec. III-A, Fig. 2): V valid samples per block, block count."""
    assert n_ov % 2 == 0 and 0 <= n_ov < n_block
    V = n_block - n_ov
    return V, -(-L // V)


def ols_block_input(field: np.ndarray, b: int, n_block: int, n_ov: int) -> np.ndarray:
    """Samples [b V - N_ov/2, b V - N_ov/2 + N) of the periodic input (wrapping circularly)."""
    L = field.shape[0]
    V = n_block - n_ov
    idx = np.mod(b * V - n_ov // 2 + np.arange(n_block), L)
    return field[idx, :]


def dbp_mode_b(field: np.ndarray, p: ChainParams, n_fft: int, overlap: int,
               blocks=None) -> np.ndarray:
    """Mode B: overlap-and-save blocks of N = n_sb * n_fft samples, N_ov = n_sb * overlap.

    Each block runs the full chain; the middle V = N - N_ov samples are kept (N_ov/2 dropped on
    each side); the last block's valid part is truncated to the sequence length.  With
    ``blocks`` (an iterable of block indices) only those blocks are computed and the other
    output samples are left as NaN (used to check sampled outputs of large workloads).
    """
    field = np.asarray(field, dtype=np.complex128)
    L = field.shape[0]
    N = p.n_sb * n_fft
    n_ov = p.n_sb * overlap
    V, n_blocks = ols_geometry(L, N, n_ov)
    out = np.full((L, 2), np.nan + 0j, dtype=np.complex128)
    todo = range(n_blocks) if blocks is None else blocks
    for b in todo:
        y = cbessfm_block(ols_block_input(field, b, N, n_ov), p)
        n_keep = min(V, L - b * V)
        out[b * V: b * V + n_keep] = y[n_ov // 2: n_ov // 2 + n_keep]
    return out


# ---------------------------------------------------------------------------------------------
# Mode S: per-step streaming.  The operator sequence of the chain,
#   G((1 - rho) L) NLPR_0 G(L) NLPR_1 G(L) ... NLPR_{N_st - 1} G(rho L),
# is cut into one pass per step, pass s = [G_a(s)] NLPR_s G_b(s) with G_a(0) = G((1 - rho) L)
# (none after), G_b(s) = G(L) and G_b(N_st - 1) = G(rho L).  Every pass runs its own
# overlap-and-save over the full band (FFT, DEMUX, subband IFFTs, NLPR, FFTs, MUX, IFFT) and the
# field is stored between passes, so a pass's overlap needs to cover one step's memory only.
# ---------------------------------------------------------------------------------------------

def _pass_block(u: np.ndarray, p: ChainParams, s: int) -> np.ndarray:
    """Pass s of mode S on one circular block u (N, 2)."""
    N = u.shape[0]
    n_sb = p.n_sb
    _, b = subband_bins(N, n_sb)
    freq = b * (p.sample_rate / N)
    Ls = p.step_length
    X = demux(np.fft.fft(u, axis=0), n_sb)
    if s == 0:
        X = X * gvd_factor(p.beta2, (1.0 - p.ratio) * Ls, freq)[..., None]
    us = nlpr(subband_to_time(X, N), p.taps[s], p.per_pol)
    X = time_to_subband(us, N)
    dz = Ls if s < p.n_st - 1 else p.ratio * Ls
    X = X * gvd_factor(p.beta2, dz, freq)[..., None]
    return np.fft.ifft(mux(X), axis=0)


def dbp_mode_s(field: np.ndarray, p: ChainParams, n_fft: int, overlap: int) -> np.ndarray:
    """Mode S: one overlap-and-save pass over the whole sequence per step (N = n_sb n_fft,
    N_ov = n_sb overlap, the middle V = N - N_ov samples kept).  With N_st = 0 it is mode B."""
    field = np.asarray(field, dtype=np.complex128)
    if p.n_st == 0:
        return dbp_mode_b(field, p, n_fft, overlap)
    L = field.shape[0]
    N = p.n_sb * n_fft
    n_ov = p.n_sb * overlap
    V, n_blocks = ols_geometry(L, N, n_ov)
    for s in range(p.n_st):
        out = np.zeros((L, 2), dtype=np.complex128)
        for b in range(n_blocks):
            y = _pass_block(ols_block_input(field, b, N, n_ov), p, s)
            n_keep = min(V, L - b * V)
            out[b * V: b * V + n_keep] = y[n_ov // 2: n_ov // 2 + n_keep]
        field = out
    return field
