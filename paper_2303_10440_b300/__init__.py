"""B300-native differentiable mesh-Fourier fluorescence renderer (deltaMic hot path).

The compute path is the in-tree CUDA library libdeltamic.so (sm_103a); this package
only marshals arguments to its C ABI (include/deltamic.h).
"""

from .api import PSF, DeltaMicError, Grid, Renderer  # noqa: F401

__all__ = ["Grid", "PSF", "Renderer", "DeltaMicError"]
