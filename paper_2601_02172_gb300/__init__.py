"""GB300-native X-FFT solver for periodic 3D linear-elastic homogenization (arXiv 2601.02172).

The compute path is the CUDA library ``libxfft.so`` (sources in ``csrc/``, C-ABI in
``include/xfft.h``); this package only builds it and marshals arguments to it.
"""
from .build import build  # noqa: F401
from .capi import Solver, XfftError, batch_effective_stiffness, lib  # noqa: F401


def effective_stiffness(solver, L, lame, scale=None):
    """Differentiable C_eff (torch) of a microstructure; see ``autograd.py``."""
    from .autograd import effective_stiffness as _f
    return _f(solver, L, lame, scale)
