"""CPU FP64 oracle for the FX spectral correlator (Prasad & Subrahmanya,
"Software Spectral Correlator for the 44-Element Ooty Radio Telescope").

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code
with the CUDA path (no kernels, headers, tables or constant generators); the
two meet only at the packed 4-bit input bytes, which a separate seeded
generator writes.

Every function is the plain definition of the quantity the paper computes,
in float64, with library primitives (a matrix product, numpy's FFT in the
self-checks) used only as whole steps:

* ``fx``   -- unpack, integer sample delays of the streaming form, direct
              DFT, gain/delay correction, cross-multiply and accumulate
              (Sec. 1 and Sec. 4 of the paper).
* ``grad`` -- closed-form gradient of the visibility loss with respect to the
              per-antenna gains and delays applied before the cross-multiply.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, brute force, invariants and
statistical expectations; none is "parity unpinned".
"""

from .fx import (  # noqa: F401
    baseline_index,
    baseline_pairs,
    correction_factors,
    correlate,
    delay_samples,
    dft_matrix,
    spectra,
    unpack,
    visibilities,
    visibilities_channels,
    full_visibility_matrix,
)
from .grad import loss, loss_and_grad  # noqa: F401
