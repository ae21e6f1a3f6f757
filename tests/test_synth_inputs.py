"""The seeded input recipes (no GPU): determinism, the stated volume fractions and shapes, and
the separation that keeps every tet away from two interfaces."""
import math

import numpy as np

import synth
from synth.geometry import _min_gap, _periodic_diff


def test_spheres27_recipe():
    w1 = synth.make_workload("spheres27")
    w2 = synth.make_workload("spheres27")
    assert np.array_equal(w1["L"], w2["L"])
    info = w1["info"]
    r = np.asarray(info["radii"])
    c = np.asarray(info["centers"])
    assert len(r) == 27
    # one common factor brings the drawn radii (U[0.06, 0.12]) to exactly 20 % volume
    assert abs(4.0 / 3.0 * math.pi * float(np.sum(r ** 3)) - 0.20) < 1e-12
    assert np.all(r / info["factor"] >= 0.06 - 1e-15) and np.all(r / info["factor"] <= 0.12 + 1e-15)
    gap = _min_gap(w1["n"], w1["length"])
    for i in range(27):
        for j in range(i + 1, 27):
            d = _periodic_diff(c[i], c[j], np.ones(3))
            assert math.sqrt(float(d @ d)) >= r[i] + r[j] + gap


def test_ellipsoids40_recipe():
    w = synth.make_workload("ellipsoids40")
    info = w["info"]
    assert info["count"] == 40 and abs(info["vf"] - 0.25) < 1e-15
    v_each = 0.25 / 40
    for inc in info["inclusions"]:
        a, b, c = inc["semi"]
        assert a >= b >= c > 0.0 and a / c <= 3.0 + 1e-12
        assert abs(4.0 / 3.0 * math.pi * a * b * c - v_each) < 1e-15
        R = np.asarray(inc["R"])
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-12) and abs(np.linalg.det(R) - 1.0) < 1e-12
    # at every node at most one inclusion comes within one voxel diagonal (so no tet, whose
    # vertices all lie within one voxel diagonal of an interface crossing it, sees two)
    n = w["n"]
    gap = _min_gap(n, w["length"])
    near = np.zeros(n, dtype=np.int32)
    for inc in info["inclusions"]:
        near += synth.ellipsoids_levelset(n, [inc]) < gap
    assert near.max() == 1
    assert w["scale"].dtype == np.float32 and 0.8 <= w["scale"].min() and w["scale"].max() <= 1.2
    # the union is the minimum of the inclusions' level sets
    assert np.array_equal(w["L"] < 0, synth.ellipsoids_levelset(n, info["inclusions"]) < 0)


def test_hashin_inputs():
    Ls, ph, ell = synth.hashin_neutral_inclusion(16)
    assert Ls.shape == (2, 16, 16, 16) and ell == (16.0, 16.0, 16.0)
    for (lam, mu), K in zip(ph, synth.HASHIN["bulk_MPa"]):
        assert abs(lam + 2.0 * mu / 3.0 - K) < 1e-12 * K
        assert abs(lam / (2.0 * (lam + mu)) - 0.25) < 1e-12
    # innermost first: negative inside the inclusion, and inside the coating's outer sphere
    assert Ls[0].min() < 0 and np.all(Ls[0] >= Ls[1])


def test_hashin_contrast_moduli_reproduce_the_paper_table():
    """The neutrality condition of the coated sphere (composite-sphere bulk modulus = matrix
    modulus 1) gives, at K_i / K_c = 10, the paper's printed coating and inclusion moduli
    (0.808024 and 8.080240 MPa, Sec. 4.2 table); K_i / K_c is the ratio asked for."""
    Ki, Kc, Km = synth.hashin_neutral_moduli(10.0)
    # (the table's six digits: K_c = 0.8080241, K_i = 8.080241 to 1e-6, printed 8.080240)
    assert abs(Kc - 0.808024) < 1e-6 and abs(Ki - 8.080240) < 2e-6 and Km == 1.0
    for ratio in (1e-5, 1e-1, 1e3, 1e5):
        Ki, Kc, Km = synth.hashin_neutral_moduli(ratio)
        assert abs(Ki / Kc - ratio) < 1e-12 * ratio and Kc > 0
