"""Seeded periodic microstructure generators producing nodal level sets.

Conventions shared by every consumer:

* The cell is ``[0, l1] x [0, l2] x [0, l3]``; the grid has ``n = (N1, N2, N3)`` voxels per
  axis and the same number of periodic nodes; node ``(i, j, k)`` sits at ``(i h1, j h2, k h3)``
  with ``h_a = l_a / N_a``.
* Level-set arrays have shape ``(N1, N2, N3)`` in C order (the last axis is the fastest).
* ``L < 0`` marks the inclusion phase, ``L > 0`` the matrix phase (Sec. 2.1, level-set
  definition of the two phases).
* Multi-inclusion level sets are the pointwise minimum of the individual ones; the random
  sequential addition keeps every pair of inclusions at least ``gap`` apart on the grid so that
  no P1 tetrahedron is crossed by two interfaces (the method assumes one interface per element,
  Sec. 1.2).

Everything here is input preparation: RNG draws, signed distances and rejection sampling.
All random numbers come from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np


def node_coords(n, length=(1.0, 1.0, 1.0)):
    """Return the three coordinate arrays (broadcastable to ``n``) of the periodic nodes."""
    n = tuple(int(v) for v in n)
    h = [length[a] / n[a] for a in range(3)]
    x = (np.arange(n[0]) * h[0]).reshape(-1, 1, 1)
    y = (np.arange(n[1]) * h[1]).reshape(1, -1, 1)
    z = (np.arange(n[2]) * h[2]).reshape(1, 1, -1)
    return x, y, z


def _periodic_diff(a, c, ell):
    d = a - c
    return d - ell * np.round(d / ell)


def sphere_levelset(n, center, radius, length=(1.0, 1.0, 1.0)):
    """Signed distance ``|x - c|_periodic - r`` sampled at the nodes."""
    x, y, z = node_coords(n, length)
    dx = _periodic_diff(x, center[0], length[0])
    dy = _periodic_diff(y, center[1], length[1])
    dz = _periodic_diff(z, center[2], length[2])
    return np.sqrt(dx * dx + dy * dy + dz * dz) - radius


def coated_sphere_levelsets(n, center, r_inclusion, r_coating, length=(1.0, 1.0, 1.0)):
    """Two level sets of a coated sphere, innermost first (shape (2,) + n): negative inside
    the inclusion, and inside the coating's outer sphere.  With the phase of a point taken from
    the first negative level set, the phases are inclusion, coating, matrix."""
    return np.stack([sphere_levelset(n, center, r_inclusion, length),
                     sphere_levelset(n, center, r_coating, length)])


# Hashin's neutral inclusion (Sec. 4.2, table "Geometry and parameters"): a 16 um cubic cell,
# a coated sphere in its centre with inclusion radius 6e/5 um and coating radius 2 pi um, bulk
# moduli 8.080240 / 0.808024 / 1.0 MPa (inclusion / coating / matrix), Poisson's ratio 0.25 in
# all phases; load eps_bar = I.  The composite-sphere formula gives K_eff = K_matrix.
HASHIN = {
    "cell_um": 16.0,
    "r_inclusion_um": 6.0 * math.e / 5.0,
    "r_coating_um": 2.0 * math.pi,
    "bulk_MPa": (8.080240, 0.808024, 1.0),
    "poisson": 0.25,
}


def hashin_neutral_inclusion(N):
    """Level sets (2, N, N, N), phases [(lambda, mu)] * 3 (inclusion, coating, matrix) and the
    cell edge lengths of Hashin's neutral inclusion on an N^3 grid."""
    ell = (HASHIN["cell_um"],) * 3
    c = tuple(x / 2.0 for x in ell)
    Ls = coated_sphere_levelsets((N, N, N), c, HASHIN["r_inclusion_um"], HASHIN["r_coating_um"], ell)
    phases = [lame_from_K_nu(K, HASHIN["poisson"]) for K in HASHIN["bulk_MPa"]]
    return Ls, phases, ell


def hashin_neutral_moduli(ratio, K_matrix=1.0, poisson=0.25):
    """Bulk moduli (inclusion, coating, matrix) of a neutral coated sphere with K_i / K_c =
    ``ratio`` (the contrast study of Sec. 4.2): the composite sphere's bulk modulus
    K* = K_c + c (K_i - K_c) / (1 + (1 - c)(K_i - K_c) / (K_c + 4 mu_c / 3)), c = (r_i / r_c)^3
    (Hashin 1962), equals K_matrix.  With a common Poisson ratio mu_c = a K_c,
    a = 3 (1 - 2 nu) / (2 (1 + nu)), and K* is K_c times a function of the ratio alone."""
    c = (HASHIN["r_inclusion_um"] / HASHIN["r_coating_um"]) ** 3
    a = 3.0 * (1.0 - 2.0 * poisson) / (2.0 * (1.0 + poisson))
    q = ratio - 1.0
    Kc = K_matrix / (1.0 + c * q / (1.0 + (1.0 - c) * q / (1.0 + 4.0 * a / 3.0)))
    return (ratio * Kc, Kc, K_matrix)


def hashin_contrast(N, ratio):
    """Hashin's neutral inclusion on an N^3 grid with the inclusion/coating bulk-modulus ratio
    ``ratio`` (matrix K = 1, all Poisson ratios 0.25): level sets, phases, cell lengths."""
    Ls, _, ell = hashin_neutral_inclusion(N)
    phases = [lame_from_K_nu(K, HASHIN["poisson"]) for K in hashin_neutral_moduli(ratio)]
    return Ls, phases, ell


def spheres_levelset(n, centers, radii, length=(1.0, 1.0, 1.0)):
    """Minimum over spheres of the periodic signed distances."""
    L = np.full(tuple(n), np.inf)
    for c, r in zip(centers, radii):
        L = np.minimum(L, sphere_levelset(n, c, r, length))
    return L


def _min_gap(n, length):
    # one voxel diagonal (with a 1% margin): every vertex of a tetrahedron crossed by an
    # interface lies within one voxel diagonal of that interface
    h = math.sqrt(sum((length[a] / n[a]) ** 2 for a in range(3)))
    return 1.01 * h


def rsa_spheres(n, count, rmin, rmax, vf, seed, length=(1.0, 1.0, 1.0), gap=None,
                max_attempts=200000):
    """Random sequential addition of ``count`` non-overlapping spheres.

    Radii are drawn uniformly in ``[rmin, rmax]`` and then multiplied by one common factor so
    that the spheres' total volume equals ``vf`` of the cell.  Centres are uniform; a candidate
    is rejected unless its periodic distance to every placed centre is at least
    ``r_i + r_j + gap`` (default gap: two voxel diagonals).

    Returns ``(L, info)`` with ``info = {centers, radii, factor, vf}``.
    """
    rng = np.random.default_rng(seed)
    vol = float(np.prod(length))
    radii = rng.uniform(rmin, rmax, size=count)
    factor = (vf * vol / (4.0 / 3.0 * math.pi * float(np.sum(radii ** 3)))) ** (1.0 / 3.0)
    radii = np.sort(radii * factor)[::-1]
    gap = _min_gap(n, length) if gap is None else gap
    ell = np.asarray(length, dtype=float)
    centers = []
    attempts = 0
    for r in radii:
        while True:
            attempts += 1
            if attempts > max_attempts:
                raise RuntimeError("rsa_spheres: jammed; lower vf or count")
            c = rng.uniform(0.0, 1.0, size=3) * ell
            ok = True
            for cj, rj in zip(centers, radii):
                d = _periodic_diff(c, cj, ell)
                if math.sqrt(float(d @ d)) < r + rj + gap:
                    ok = False
                    break
            if ok:
                centers.append(c)
                break
    L = spheres_levelset(n, centers, radii[: len(centers)], length)
    return L, {"centers": np.array(centers), "radii": radii, "factor": factor, "vf": vf}


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def _box_indices(n, length, center, reach):
    """Node index ranges (periodic, as index arrays) of the box ``center +- reach``."""
    idx = []
    for a in range(3):
        h = length[a] / n[a]
        lo = int(math.floor((center[a] - reach) / h))
        hi = int(math.ceil((center[a] + reach) / h))
        if hi - lo + 1 >= n[a]:
            idx.append(np.arange(n[a]))
        else:
            idx.append(np.arange(lo, hi + 1) % n[a])
    return idx


def _ellipsoid_levelset_box(n, length, center, R, semi, ix, iy, iz):
    """Ellipsoid level set on a box: ``f / |grad f|`` with ``f = ||diag(1/semi) R^T (x-c)|| - 1``."""
    ell = np.asarray(length, dtype=float)
    h = ell / np.asarray(n)
    X = _periodic_diff(ix.reshape(-1, 1, 1) * h[0], center[0], ell[0])
    Y = _periodic_diff(iy.reshape(1, -1, 1) * h[1], center[1], ell[1])
    Z = _periodic_diff(iz.reshape(1, 1, -1) * h[2], center[2], ell[2])
    # body-frame coordinates: xb = R^T (x - c); f = ||xb||_A - 1 and its gradient norm
    q = 0.0
    g2 = 0.0
    for a in range(3):
        xb = R[0, a] * X + R[1, a] * Y + R[2, a] * Z
        q = q + (xb / semi[a]) ** 2
        g2 = g2 + (xb / semi[a] ** 2) ** 2
    nrm = np.sqrt(q)
    grad = np.sqrt(g2) / np.maximum(nrm, 1e-300)
    # first-order signed distance f / |grad f| (exact for spheres, zero set unchanged)
    return (nrm - 1.0) / np.maximum(grad, 1.0 / float(np.max(semi)))


def rsa_ellipsoids(n, count, vf, seed, aspect=(1.0, 3.0), length=(1.0, 1.0, 1.0), gap=None,
                   spheres_only=False, max_attempts=20000):
    """Random sequential addition of randomly oriented ellipsoids.

    Semi-axes ``a >= b >= c`` with ``a/c`` uniform in ``aspect`` and ``b/c`` uniform in
    ``[1, a/c]``; every inclusion gets the volume ``vf |Y| / count``.  The level set of one
    ellipsoid is the first-order signed distance ``f / |grad f|`` of the implicit function
    ``f = ||A^{-1/2} R^T (x - c)|| - 1`` (same zero set, unit slope at the surface).  A node
    test ``L_new < gap and L_old < gap`` with ``gap`` of one voxel diagonal rejects every
    candidate that would share a tetrahedron (all of whose vertices lie within one voxel
    diagonal of the surface it crosses) with an earlier inclusion.  ``spheres_only`` forces
    ``a = b = c``.

    Returns ``(L, info)``; ``info['vf']`` is the analytic volume fraction actually placed.
    """
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    vol = float(np.prod(length))
    gap = _min_gap(n, length) if gap is None else gap
    v_each = vf * vol / count
    free = None
    L = np.full(n, np.inf)
    placed = []
    attempts = 0
    while len(placed) < count:
        attempts += 1
        if attempts > max_attempts:
            break
        if spheres_only:
            ratios = np.ones(3)
        else:
            ac = rng.uniform(aspect[0], aspect[1])
            bc = rng.uniform(1.0, ac)
            ratios = np.array([ac, bc, 1.0])
        cmin = (v_each / (4.0 / 3.0 * math.pi * float(np.prod(ratios)))) ** (1.0 / 3.0)
        semi = ratios * cmin
        R = np.eye(3) if spheres_only else _random_rotation(rng)
        center = rng.uniform(0.0, 1.0, size=3) * np.asarray(length)
        if placed and attempts % 2 == 0:
            # every other candidate: draw the centre among nodes that are free enough for the
            # inscribed ball, jittered inside the voxel (speeds up placement near jamming)
            if free is None or attempts % 64 == 0:
                free = np.flatnonzero(L.ravel() > 0.5 * float(v_each) ** (1.0 / 3.0) + gap)
            if free.size:
                node = np.unravel_index(int(free[rng.integers(0, free.size)]), n)
                hh = np.asarray(length, dtype=float) / np.asarray(n)
                center = (np.asarray(node) + rng.uniform(0.0, 1.0, size=3)) * hh
        # cheap pre-checks against placed inclusions: inscribed balls that overlap reject,
        # circumscribed balls that stay apart need no node test
        near = False
        reject = False
        for p in placed:
            d = _periodic_diff(center, p["center"], np.asarray(length, dtype=float))
            dist = math.sqrt(float(d @ d))
            if dist < float(semi[2] + p["semi"][2]):
                reject = True
                break
            if dist < float(semi[0] + p["semi"][0]) + gap:
                near = True
        if reject:
            continue
        ix, iy, iz = _box_indices(n, length, center, float(semi[0]) + 2.0 * gap)
        Lc = _ellipsoid_levelset_box(n, length, center, R, semi, ix, iy, iz)
        sub = L[np.ix_(ix, iy, iz)]
        if near and np.any((Lc < gap) & (sub < gap)):
            continue
        L[np.ix_(ix, iy, iz)] = np.minimum(sub, Lc)
        free = None
        placed.append({"center": center, "R": R, "semi": semi})
    # nodes outside every bounding box keep +inf; give them a finite positive value
    finite = np.isfinite(L)
    if not np.all(finite):
        big = float(np.max(L[finite])) if np.any(finite) else 1.0
        L[~finite] = max(big, gap)
    vf_placed = len(placed) * v_each / vol
    return L, {"inclusions": placed, "vf": vf_placed, "count": len(placed)}


def ellipsoids_levelset(n, inclusions, length=(1.0, 1.0, 1.0)):
    """Level set of already placed ellipsoids (the ``inclusions`` list returned by
    :func:`rsa_ellipsoids`) sampled on another grid ``n``."""
    n = tuple(int(v) for v in n)
    L = np.full(n, np.inf)
    for inc in inclusions:
        semi = np.asarray(inc["semi"], dtype=float)
        ix, iy, iz = _box_indices(n, length, inc["center"], float(semi[0]) + 4.0 * _min_gap(n, length))
        Lc = _ellipsoid_levelset_box(n, length, inc["center"], inc["R"], semi, ix, iy, iz)
        L[np.ix_(ix, iy, iz)] = np.minimum(L[np.ix_(ix, iy, iz)], Lc)
    finite = np.isfinite(L)
    if not np.all(finite):
        L[~finite] = float(np.max(L[finite])) if np.any(finite) else 1.0
    return L


def rsa_fibers(n, count, radius, seed, length=(1.0, 1.0, 1.0), gap=None, max_attempts=20000):
    """Straight periodic cylinders along randomly chosen coordinate axes.

    A fiber along axis ``a`` is the set of points whose periodic distance, in the plane
    normal to ``a``, to its axis point is below ``radius``.  Two fibers along the same axis
    need transverse separation ``2 r + gap``; fibers along different axes ``a != b`` need
    separation ``2 r + gap`` along the third axis.  Placement stops when the candidate budget
    is spent (the packing jams); ``info['vf']`` reports the reached volume fraction.
    """
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    ell = np.asarray(length, dtype=float)
    gap = _min_gap(n, length) if gap is None else gap
    fibers = []
    attempts = 0
    while len(fibers) < count and attempts < max_attempts:
        attempts += 1
        axis = int(rng.integers(0, 3))
        p = rng.uniform(0.0, 1.0, size=3) * ell
        ok = True
        for (ax2, p2) in fibers:
            if ax2 == axis:
                others = [a for a in range(3) if a != axis]
                d = _periodic_diff(p[others], p2[others], ell[others])
                if math.sqrt(float(d @ d)) < 2 * radius + gap:
                    ok = False
                    break
            else:
                third = 3 - axis - ax2
                d = abs(float(_periodic_diff(p[third], p2[third], ell[third])))
                if d < 2 * radius + gap:
                    ok = False
                    break
        if ok:
            fibers.append((axis, p))
    x, y, z = node_coords(n, length)
    coords = (x, y, z)
    L = np.full(n, np.inf)
    for axis, p in fibers:
        others = [a for a in range(3) if a != axis]
        d0 = _periodic_diff(coords[others[0]], p[others[0]], ell[others[0]])
        d1 = _periodic_diff(coords[others[1]], p[others[1]], ell[others[1]])
        L = np.minimum(L, np.broadcast_to(np.sqrt(d0 * d0 + d1 * d1) - radius, n))
    vf = len(fibers) * math.pi * radius ** 2 * 1.0
    return np.ascontiguousarray(L), {"fibers": fibers, "vf": vf, "count": len(fibers)}


def laminate_levelset(n, normal=(1, 2, 3), offset=0.1234567, fraction=0.5):
    """Signed distance of a periodic laminate on the unit cube.

    With the integer normal ``m`` the phase function depends on ``t = m . x`` only and is
    periodic on the unit cube.  Layer ``-`` occupies ``frac(t - offset) in (0, fraction)``;
    the returned value is the signed distance ``+-dist_t / |m|`` to the nearest interface
    plane (negative inside layer ``-``).
    """
    m = np.asarray(normal, dtype=float)
    x, y, z = node_coords(n)
    t = m[0] * x + m[1] * y + m[2] * z
    s = np.mod(t - offset, 1.0)
    inside = s < fraction
    d_in = np.minimum(s, fraction - s)
    d_out = np.minimum(s - fraction, 1.0 - s)
    L = np.where(inside, -d_in, d_out) / np.linalg.norm(m)
    return np.ascontiguousarray(np.broadcast_to(L, tuple(n)).astype(np.float64))


def voxel_scale(n, seed, lo=0.8, hi=1.2):
    """Per-voxel modulus scale field, iid uniform in ``[lo, hi]``, float32, shape ``n``."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(n)).astype(np.float32)


def lame_from_K_nu(K, nu):
    """Return ``(lambda, mu)`` of an isotropic material from its bulk modulus and Poisson ratio."""
    mu = 3.0 * K * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu))
    return (float(K - 2.0 * mu / 3.0), float(mu))


def lame_from_E_nu(E, nu):
    """Return ``(lambda, mu)`` of an isotropic material from Young's modulus and Poisson ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return (float(lam), float(mu))


def _unit_strains(count):
    return [np.eye(6)[k].copy() for k in range(count)]


def make_workload(name, n=None, seed=None):
    """Build one of the named synthetic workloads.

    Returns a dict with keys ``n``, ``length``, ``L`` (float64, C order), ``lame_minus`` (the
    ``L < 0`` inclusion phase), ``lame_plus`` (the ``L > 0`` matrix phase), ``scale``
    (float32 or None), ``eps`` (list of Mandel strain 6-vectors), ``info``.
    """
    spec = WORKLOADS[name]
    return spec(n=n, seed=seed)


def _single_sphere(n=None, seed=None):
    n = (16, 16, 16) if n is None else tuple(n)
    L = sphere_levelset(n, (0.5, 0.5, 0.5), 0.3)
    return {"n": n, "length": (1.0, 1.0, 1.0), "L": L,
            "lame_minus": lame_from_E_nu(10.0, 0.3), "lame_plus": lame_from_E_nu(1.0, 0.3),
            "scale": None, "eps": _unit_strains(1), "info": {"geometry": "sphere r=0.3"}}


def _spheres27(n=None, seed=None):
    n = (64, 64, 64) if n is None else tuple(n)
    seed = 2 if seed is None else seed
    L, info = rsa_spheres(n, 27, 0.06, 0.12, 0.20, seed)
    return {"n": n, "length": (1.0, 1.0, 1.0), "L": L,
            "lame_minus": lame_from_E_nu(100.0, 0.2), "lame_plus": lame_from_E_nu(1.0, 0.3),
            "scale": None, "eps": _unit_strains(6), "info": info}


def _ellipsoids40(n=None, seed=None):
    n = (128, 128, 128) if n is None else tuple(n)
    seed = 4 if seed is None else seed
    L, info = rsa_ellipsoids(n, 40, 0.25, seed)
    return {"n": n, "length": (1.0, 1.0, 1.0), "L": L,
            "lame_minus": lame_from_E_nu(50.0, 0.2), "lame_plus": lame_from_E_nu(1.0, 0.3),
            "scale": voxel_scale(n, seed + 1000), "eps": _unit_strains(6), "info": info}


def _fibers60(n=None, seed=None):
    n = (256, 256, 256) if n is None else tuple(n)
    seed = 5 if seed is None else seed
    L, info = rsa_fibers(n, 60, 0.04, seed)
    return {"n": n, "length": (1.0, 1.0, 1.0), "L": L,
            "lame_minus": lame_from_E_nu(100.0, 0.2), "lame_plus": lame_from_E_nu(1.0, 0.3),
            "scale": None, "eps": _unit_strains(6), "info": info}


def _laminate(n=None, seed=None):
    n = (384, 384, 384) if n is None else tuple(n)
    L = laminate_levelset(n)
    return {"n": n, "length": (1.0, 1.0, 1.0), "L": L,
            "lame_minus": lame_from_E_nu(100.0, 0.2), "lame_plus": lame_from_E_nu(1.0, 0.3),
            "scale": None, "eps": _unit_strains(6),
            "info": {"normal": (1, 2, 3), "offset": 0.1234567, "fraction": 0.5}}


def batch_uneven(count=16, seed=3, sizes=(32, 48, 64, 80, 96)):
    """The multi-microstructure batch: uneven grids, spheres or ellipsoids, random contrast."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        N = int(rng.choice(sizes))
        vf = float(rng.uniform(0.1, 0.3))
        contrast = float(np.exp(rng.uniform(np.log(10.0), np.log(1000.0))))
        ell = bool(rng.integers(0, 2))
        nincl = int(rng.integers(4, 12))
        sub_seed = int(rng.integers(0, 2 ** 31 - 1))
        L, info = rsa_ellipsoids((N, N, N), nincl, vf, sub_seed, spheres_only=not ell)
        out.append({"n": (N, N, N), "length": (1.0, 1.0, 1.0), "L": L,
                    "lame_minus": lame_from_E_nu(contrast, 0.2),
                    "lame_plus": lame_from_E_nu(1.0, 0.3), "scale": None,
                    "eps": _unit_strains(6), "info": dict(info, contrast=contrast)})
    return out


WORKLOADS = {
    "single_sphere": _single_sphere,
    "spheres27": _spheres27,
    "ellipsoids40": _ellipsoids40,
    "fibers60": _fibers60,
    "laminate": _laminate,
}
