"""GB300-native X-FFT solver for periodic 3D linear-elastic homogenization (arXiv 2601.02172).

The compute path is the CUDA library ``libxfft.so`` (sources in ``csrc/``, C-ABI in
``include/xfft.h``); this package only builds it and marshals arguments to it.
"""
from .build import build  # noqa: F401
from .capi import Solver, XfftError, lib  # noqa: F401
