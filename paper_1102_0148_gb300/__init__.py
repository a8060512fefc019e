"""gbcorr: an FX spectral correlator for one GB300 (sm_103a).

The method is Prasad & Subrahmanya's software spectral correlator for the
44-element Ooty Radio Telescope: a per-antenna real FFT (the F-engine)
followed by a per-channel cross-multiply-and-accumulate over every antenna
pair (the X-engine).  All compute runs in hand-written CUDA kernels behind
the C ABI declared in ``include/corr.h``; ``corr`` is the thin Python binding.

Importing this package loads nothing native; ``from paper_1102_0148_gb300
import corr`` loads the shared library and fails loudly if it is missing.
"""

__all__ = ["corr", "synth", "build"]
