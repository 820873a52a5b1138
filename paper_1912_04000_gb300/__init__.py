"""GB300 spectral path tracer: one wavelength band per Monte Carlo path.

Hot path in hand-written CUDA for sm_103a behind a C ABI
(include/spectral_rt.h); this package is the thin Python binding plus the
seeded scene generators.
"""
from . import scenes  # noqa: F401
from ._native import XYZ_BF16, XYZ_BF16X3, XYZ_FP64, RtError  # noqa: F401


def Renderer(*args, **kwargs):
    from .renderer import Renderer as _R
    return _R(*args, **kwargs)
