"""GB300 (sm_103a) implementation of the wave-equation hot path of
"Robust Full Waveform Inversion with deep Hessian deblurring" (arXiv 2403.17518).

The compute path is the CUDA library ``libdhfwi.so`` (C ABI in
``include/dhfwi.h``); :mod:`.ops` binds it for PyTorch tensors.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Context", "FWIMisfit", "GeomArgs", "DhfwiError", "DHFWI_ABS", "DHFWI_REL"):
        from . import ops

        return getattr(ops, name)
    raise AttributeError(name)
