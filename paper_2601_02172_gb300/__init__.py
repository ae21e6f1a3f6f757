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


def solve(L, lame_minus, lame_plus, eps_bar, scale=None, precision="fp64", length=(1.0, 1.0, 1.0),
          tol=None, voxel_stress=False, device=None, phases=None):
    """One-call solve of the cell problem on the grid of the nodal level set ``L`` (shape
    (n0, n1, n2)) for the Mandel strains ``eps_bar`` (k x 6): displacement fluctuation (standard
    and unscaled enriched parts), mean stress, optionally the per-voxel stress; NumPy outputs, or
    CUDA tensors when ``device`` is given.  ``lame_minus`` / ``lame_plus`` are (lambda, mu) of the
    L < 0 and L > 0 phases.  Several interfaces: ``L`` of shape (K, n0, n1, n2) and ``phases``
    the K + 1 pairs (lambda, mu) (``lame_minus`` / ``lame_plus`` are then ignored)."""
    n = tuple(int(v) for v in (L.shape[1:] if phases is not None else L.shape))
    kw = {} if tol is None else {"tol": tol}
    s = Solver(n, length, precision=precision, **kw)
    try:
        if phases is not None:
            s.set_microstructure_phases(L, phases, scale)
        else:
            s.set_microstructure(L, lame_minus, lame_plus, scale)
        return s.solve(eps_bar, u=True, voxel_stress=voxel_stress, device=device)
    finally:
        s.close()
