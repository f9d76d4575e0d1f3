"""CPU oracle for streaming method-of-snapshots DMD (arXiv 1612.07875).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its CPU legs ``cpu_baseline`` and ``cpu_streaming`` and its
``--impl reference`` arm) may
import, call, link or execute anything under ``oracle/``. The product package
``paper_1612_07875_gb300`` never imports it, and the oracle imports nothing
from the product package except the seeded input generators, which hold none
of the method's arithmetic.

What the oracle computes, after every streamed snapshot, from scratch:

* the window's inner-product matrix G = W^H W (method of snapshots, Sec. 2.1,
  Eq. 3 left-hand side; the streaming form Eq. 12a-b gives the same entries),
  in FP64 / complex128 for float data and exactly in int64 for 8-bit data;
* the exact DMD of the window (Sec. 2.2, Eqs. 5-9 and Algorithms 1-2):
  sym-eig of X^H X, sigma, V, A~ = Sigma^-1 V^H X^H X' V Sigma^-1, eig(A~),
  Phi = X' V Sigma^-1 W;
* the mode amplitudes from POD coefficients (Sec. 3.3, Eq. 14a-e) and the
  background mode of Algorithm 3.

``native.StreamingCPU`` (C, ``stream_cpu.c``) is not a parity reference but the
timed streaming CPU baseline: the streaming Gram update of Eq. 12a-b run on
the host cores, pinned to the brute-force Gram of its ring.

Equation numbers follow the order of the equations in the paper's LaTeX
source: (1) X, (2) X = U Sigma V*, (3) X*X V = V Lambda, (4) U = X V Sigma^-1,
(5) X', (6) A = X' X^+, (7) A~ = U* X' V Sigma^-1, (8) A~ W = W Lambda,
(9) Phi = X' V Sigma^-1 W, (10) X = L + S, (11) background/foreground split,
(12a-b) the streaming Gram, (13) b = Phi^+ x_1, (14a-e) b from POD coefficients.

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: brute-force sums, numpy.linalg.svd, closed forms, planted systems,
pseudo-inverse operators and Parseval's identity.
"""

from .gram import (gram_dense, cross_gram, gram_u8, gram_u8_cols, dot_u8, sparse_inner,
                   gram_sparse, densify_sparse)
from .dmd import (RANK_RTOL_FACTOR, numerical_rank, mos_svd, exact_dmd, dmd_from_gram,
                  DMDResult, pod_amplitudes, lstsq_amplitudes,
                  background_index, background_column, reconstruct, foreground_column,
                  pod_modes, slow_modes, slow_background_column, slow_foreground_column,
                  fourier_dmd, fourier_support, fourier_phi_rows)
from .stream import StreamOracle

__all__ = [
    "gram_dense", "cross_gram", "gram_u8", "gram_u8_cols", "dot_u8", "sparse_inner",
    "gram_sparse", "densify_sparse", "RANK_RTOL_FACTOR", "numerical_rank",
    "mos_svd", "exact_dmd", "dmd_from_gram", "DMDResult", "pod_amplitudes", "lstsq_amplitudes",
    "background_index", "background_column", "reconstruct", "foreground_column", "pod_modes",
    "slow_modes", "slow_background_column", "slow_foreground_column", "fourier_dmd",
    "fourier_support", "fourier_phi_rows", "StreamOracle",
]
