"""GB300-native perspective-correct 3D Gaussian splatting with hybrid
transparency (arXiv 2410.08129).

The rendering path runs entirely in hand-written sm_103a CUDA kernels behind a
C-ABI library (``include/htgs.h``); this package is the thin Python binding
over it. Importing the package does not load the CUDA library; the first call
into the binding does, and it raises if the library is missing.
"""
from . import scenes  # noqa: F401  (seeded input generators; no method arithmetic)

__all__ = ["scenes"]
