"""The N' = 1024 DEMUX/MUX twiddle scheme on the host, in float32: W_N^(K r) for r = 1 .. 4 as
powers of W_N^K, itself the product of two unit-modulus table values (W_N^(K_0) and the slot's
row-1 factor), stays within a few float roundings of the exact twiddle.  This bounds what the
scheme adds to the chain's error (the GPU parity suite checks the kernel itself)."""
import numpy as np


def _unit32(num, den):
    """exp(-2 pi i num / den) rounded to complex64 (the tables are built in FP64 and rounded)."""
    return np.exp(-2j * np.pi * (np.asarray(num, dtype=np.float64) % den) / den).astype(np.complex64)


def test_powers_of_a_gathered_twiddle_stay_within_a_few_roundings():
    n_sb, NP = 5, 1024
    N = n_sb * NP
    TPF, E = 32, 32
    worst = 0.0
    for gi in range(n_sb):
        ci = -N // 2 + gi * NP + NP // 2
        for j in range(TPF):
            K0 = (ci + j) % N
            wk0 = _unit32(K0, N)
            for t in range(E):
                kap = j + TPF * t
                K = (ci + (kap if kap < NP // 2 else kap - NP)) % N
                # slot t's row-1 factor, as the plan tables hold it
                td1 = _unit32(TPF * t - (NP if t >= E // 2 else 0), N)
                w1 = np.complex64(wk0 * td1)
                w = w1
                for r in range(1, n_sb):
                    exact = np.exp(-2j * np.pi * ((K * r) % N) / N)
                    worst = max(worst, abs(complex(w) - exact))
                    w = np.complex64(w * w1)
    # float32 spacing at 1 is 1.19e-7 and the chain is at most four products deep: every
    # slot of every thread of the c2 shape stays below 5.3e-7 (host emulation without FMA)
    assert worst < 6e-7, worst
