"""FP64 CPU oracle for CB-ESSFM digital backpropagation -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy implementations of what the GPU hot path computes, written
from the paper's description (Sec. III-A and Figs. 2-4 for the algorithm, Sec. III-C for the
splitting ratio, Eq. (NLPR-multiband-2pol) for the nonlinear phase).  It shares no code with the
CUDA library and never imports it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; the product path never
does.

Modules
-------
``dbp``       the CB-ESSFM chain on one circular block, mode U (whole sequence) and mode B
              (overlap-and-save), plus the subband DEMUX/MUX used by it.
``adjoint``   FP64 reverse-mode gradient of the chain (taps, splitting ratio, input).
``channel``   fine-step split-step Fourier simulation of the Manakov equation (input generator).
``evaluate``  matched filter, 1 sample/symbol, mean-phase removal, SNR (Sec. IV-A).
``coeffs``    analytic CB-ESSFM coefficients: closed-form Volterra kernel and the double
              integral of its diagonal response (Sec. II-D).

Parity pins live in ``tests/test_oracle_*.py``.  Every function here is pinned by at least one
check that is not a re-typing of its own formula; see the test module docstrings.
"""
from . import dbp, channel, evaluate, adjoint, coeffs  # noqa: F401
