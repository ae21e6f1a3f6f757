"""Oracle pins of the P1 baseline (enrichment off, the discretization table of Sec. 4.1) and of
the Barzilai-Borwein step rules (Sec. 2.3 cites the scheme without its formula).

P1: a laminate whose interfaces lie on node planes has a piecewise-affine solution that the
voxel-segmented P1 space contains, so its C_eff is the closed form; with a tilted interface P1
is only first-order accurate (unlike X-FEM, which stays exact there) and C_eff lies between the
Voigt and Reuss bounds of its own voxel phase fractions.  PCG equals the direct solve.

Barzilai-Borwein: every step rule reaches the direct solution; where the preconditioned operator
is a multiple c of the identity (a homogeneous cell whose stiffness is c times the reference
material) every rule's first Barzilai-Borwein step is the exact 1/c, so the scheme stops after
the second iteration whatever the first step was.
"""
import numpy as np
import pytest

import synth
from oracle import XFEM, iso_stiffness
from test_oracle_pins import _laminate_closed_form

LM = synth.lame_from_E_nu(10.0, 0.2)
LP = synth.lame_from_E_nu(1.0, 0.3)


def _ceff_direct(o):
    o.assemble()
    C = np.zeros((6, 6))
    for k in range(6):
        e = np.eye(6)[k]
        C[:, k] = o.mean_stress(o.solve_direct(e), e)
    return C


def test_p1_voxel_phases_follow_the_centre_value():
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    o = XFEM(L, n, lame_minus=LM, lame_plus=LP, enrichment=False)
    assert o.nX == 0 and len(o.cut_list) == 0 and not o.cut.any()
    # the centre value: trilinear interpolation of the corner values = their mean
    Ln = o.L.reshape(n)
    centre = np.zeros(n)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                centre += np.roll(Ln, (-dx, -dy, -dz), axis=(0, 1, 2)) / 8.0
    exp = np.where(centre.ravel() < 0, 0, 1)
    for t in range(6):
        assert np.array_equal(o.tet_phase[:, t], exp)


def test_p1_laminate_on_node_planes_is_exact():
    """Interfaces on node planes (normal (1,0,0), offset 1/4, 8^3): every voxel lies in one layer
    and the laminate's piecewise-affine solution is in the P1 space: C_eff = closed form, the
    same as X-FEM's."""
    n = (8, 8, 8)
    L = synth.laminate_levelset(n, normal=(1, 0, 0), offset=0.25, fraction=0.5)
    Cref = _laminate_closed_form((1, 0, 0), 0.5, LM, LP)
    C1 = _ceff_direct(XFEM(L, n, lame_minus=LM, lame_plus=LP, enrichment=False))
    assert np.abs(C1 - Cref).max() < 1e-12 * np.abs(Cref).max()


def test_p1_tilted_laminate_is_first_order_and_bounded():
    """A tilted laminate: X-FEM is exact (its solution lies in V_h), P1 is not: P1's error falls
    as the grid is refined; C_eff lies within the Voigt and Reuss bounds of P1's own voxel phase
    fractions (u = 0 is admissible; V_h is a subspace of H^1 on the voxelised geometry)."""
    normal = (1, 1, 2)
    Cref = _laminate_closed_form(normal, 0.5, LM, LP)
    errs = []
    for N in (8, 16):
        n = (N, N, N)
        L = synth.laminate_levelset(n, normal=normal, offset=0.137, fraction=0.5)
        o = XFEM(L, n, lame_minus=LM, lame_plus=LP, enrichment=False)
        C1 = _ceff_direct(o)
        errs.append(np.abs(C1 - Cref).max() / np.abs(Cref).max())
        f_minus = np.mean(o.tet_phase[:, 0] == 0)
        Cm, Cp = iso_stiffness(*LM), iso_stiffness(*LP)
        voigt = f_minus * Cm + (1 - f_minus) * Cp
        reuss = np.linalg.inv(f_minus * np.linalg.inv(Cm) + (1 - f_minus) * np.linalg.inv(Cp))
        Cs = 0.5 * (C1 + C1.T)
        assert np.linalg.eigvalsh(voigt - Cs).min() > -1e-12
        assert np.linalg.eigvalsh(Cs - reuss).min() > -1e-12
    # (X-FEM on the same laminate at 20^3 equals the closed form to 1e-9:
    # test_oracle_pins.test_tilted_laminate_matches_closed_form)
    assert errs[0] > 1e-3 and errs[1] < errs[0]


def test_p1_pcg_matches_direct():
    n = (10, 12, 8)
    L = np.minimum(synth.sphere_levelset(n, (0.3, 0.4, 0.5), 0.22),
                   synth.sphere_levelset(n, (0.8, 0.85, 0.2), 0.15))
    o = XFEM(L, n, lame_minus=LM, lame_plus=LP, scale=synth.voxel_scale(n, 3), enrichment=False)
    e = np.array([0.3, -0.1, 0.2, 0.05, 0.1, -0.2])
    ud = o.solve_direct(e)
    up, info = o.pcg(e, tol=1e-12, green="fft")
    assert info["converged"] and np.abs(up - ud).max() < 1e-9 * np.abs(ud).max()


@pytest.fixture(scope="module")
def sphere8():
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    o = XFEM(L, n, lame_minus=synth.lame_from_E_nu(20.0, 0.2), lame_plus=LP)
    return o


@pytest.mark.parametrize("rule,cycle", [("bb1", 1), ("bb2", 1), ("alt", 1), ("bb2e", 1), ("bb1", 3),
                                        ("bb2", 2)])
def test_bb_rules_reach_the_direct_solution(sphere8, rule, cycle):
    o = sphere8
    e = np.array([0.2, -0.1, 0.3, 0.4, -0.2, 0.1])
    ud = o.solve_direct(e)
    u, info = o.pcg(e, tol=1e-11, maxit=5000, scheme="bb", green="fft", bb_rule=rule, bb_cycle=cycle)
    assert info["converged"]
    assert np.linalg.norm(u - ud) < 1e-8 * np.linalg.norm(ud)


@pytest.mark.parametrize("rule", ["bb1", "bb2", "alt", "bb1e", "bb2e"])
def test_bb_step_is_exact_when_the_preconditioned_operator_is_scalar(rule):
    """Homogeneous cell of C = c * I_sym (lambda = 0, 2 mu = c; the reference material of P is
    I_sym): P^-1 A = c I on the standard DOFs.  From a random start with a deliberately wrong
    first step s0 = 0.3 / c the P-metric rules give the step 1/c at the second iteration, which
    zeroes the residual: two iterations.  The Euclidean rules measure du in the metric of the
    DOFs, not of P, and miss 1/c."""
    n = (6, 6, 6)
    c = 3.7
    o = XFEM(np.ones(n), n, lame_minus=(0.0, c / 2), lame_plus=(0.0, c / 2))
    rng = np.random.default_rng(5)
    u0 = rng.normal(size=o.ndof)
    u0[: 3 * o.nFE] -= np.repeat(u0[: 3 * o.nFE].reshape(3, -1).mean(1), o.nFE)
    u, info = o.pcg(np.array([0.1, 0.2, -0.3, 0.0, 0.1, 0.0]), tol=1e-13, maxit=50, scheme="bb",
                    green="fft", u0=u0,
                    step=0.3 / c, bb_rule=rule)
    if rule in ("bb1", "bb2", "alt"):
        assert info["converged"] and info["iters"] == 2, info["iters"]
    else:
        # the Euclidean metric of the DOFs is not the metric of P: the step is not 1/c
        assert info["iters"] != 2 or not info["converged"]
