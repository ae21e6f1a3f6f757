"""Plain, slow FP64 CPU oracle of the X-FFT method (arXiv 2601.02172).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA path: it
assembles the X-FEM system element by element with sub-tetrahedron quadrature, solves it with a
sparse direct solver or with the paper's linear CG (Algorithm 1), and evaluates the average
stress, the effective stiffness and its gradient.

Parity status of each function is listed in the header of ``oracle/xfem.py``.
"""
from .xfem import (  # noqa: F401
    XFEM,
    mandel_extraction,
    iso_stiffness,
    symgrad_operator,
    clip_tet,
    quad4,
    classify,
)
