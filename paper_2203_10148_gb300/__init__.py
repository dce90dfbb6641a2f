"""PiTSBiCG on GB300: Python binding of the ``libpit`` C-ABI library.

The compute path lives in ``csrc/`` (hand-written sm_103a CUDA behind the
C-ABI of ``include/pit.h``); this package only marshals arguments.  The
binding is loaded on first use, and every call fails loudly when the compiled
library is missing: there is no CPU fallback.
"""
from . import inputs  # noqa: F401  (seeded workloads; no method arithmetic)
