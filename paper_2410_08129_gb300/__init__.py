"""GB300-native perspective-correct 3D Gaussian splatting with hybrid
transparency (arXiv 2410.08129).

The rendering path runs entirely in hand-written sm_103a CUDA kernels behind a
C-ABI library (``include/htgs.h``); ``binding`` is the thin ctypes layer over
it and ``renderer`` adds workspace management and a torch.autograd.Function.
Importing the package does not load the CUDA library; the first call into the
binding does, and it raises if the library is missing.
"""
from . import scenes  # noqa: F401  (seeded input generators; no method arithmetic)

__all__ = ["scenes", "binding", "renderer", "build"]


def __getattr__(name):
    if name in ("binding", "renderer", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
