"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the CPU oracle.

This package only produces *inputs* of the X-FFT cell problem: nodal level-set samples of
periodic microstructures (spheres, ellipsoids, straight fibers, a tilted laminate), phase
moduli and per-voxel modulus-scale fields.  It holds none of the method's arithmetic
(no shape functions, no quadrature, no operators, no solvers).
"""
from .geometry import (  # noqa: F401
    node_coords,
    sphere_levelset,
    coated_sphere_levelsets,
    hashin_contrast,
    hashin_neutral_inclusion,
    hashin_neutral_moduli,
    HASHIN,
    spheres_levelset,
    rsa_spheres,
    rsa_ellipsoids,
    ellipsoids_levelset,
    batch_uneven,
    rsa_fibers,
    laminate_levelset,
    voxel_scale,
    lame_from_E_nu,
    lame_from_K_nu,
    WORKLOADS,
    make_workload,
)
