"""Pins of the oracle's several-interface setting (no GPU needed).

The paper's Sec. 4.2 solves Hashin's coated sphere: three phases, two interfaces, one interface
per element.  The oracle reads it as K level sets, the phase of a point being the index of the
first negative level set (K if none), each cut tet enriched with the modified abs of its own
interface's level set and one enrichment vector per node.  Pins:

* a three-layer laminate, whose exact solution lies in that space: C_eff = the closed-form
  laminate stiffness to rounding;
* Hashin's neutral inclusion: the composite-sphere formula fixes K_eff = K_matrix; the discrete
  bulk modulus approaches it as the grid is refined, and the enriched-DOF count at N = 16 is
  the paper's 36 %;
* a second level set that is positive everywhere changes nothing (the K = 1 system);
* two interfaces through one element are refused.
"""
import math

import numpy as np
import pytest

import synth
from oracle import XFEM, iso_stiffness
from test_oracle_pins import _laminate_closed_form


def _three_layers(N, normal, fractions, offset):
    """Level sets of a periodic three-layer laminate along ``normal``: L_0 < 0 in layer 0;
    L_1 < 0 from the middle of layer 0 to the end of layer 1 (its zero set inside layer 0 is
    hidden by L_0), so that layer 2 is the rest."""
    n = (N, N, N)
    f0, f1, _ = fractions
    L0 = synth.laminate_levelset(n, normal=normal, offset=offset, fraction=f0)
    L1 = synth.laminate_levelset(n, normal=normal, offset=offset + f0 / 2, fraction=f0 / 2 + f1)
    return np.stack([L0, L1]), n


def test_three_layer_laminate_matches_closed_form():
    """Every cut tet sees one flat interface of an affine level set and no node touches two
    interfaces, so the laminate's exact solution (affine plus kinks along both interfaces) lies
    in the discrete space: C_eff equals the closed form to rounding.  A wrong side phase, a
    dropped enrichment or the wrong level set in a cut tet all break this."""
    fr = (0.36, 0.32, 0.32)
    normal = (1, 0, 1)
    Ls, n = _three_layers(16, normal, fr, 0.137)
    ph = [synth.lame_from_E_nu(10.0, 0.2), synth.lame_from_E_nu(1.0, 0.3),
          synth.lame_from_E_nu(3.0, 0.4)]
    o = XFEM(Ls, n, phases=ph)
    # both interfaces are present: layer 0's two faces (L_0) and the 1|2 face (L_1)
    assert set(np.unique(o.cut_iface)) == {0, 1}
    assert set(np.unique(o.cut_phase[+1][o.cut_iface == 0])) == {1, 2}
    assert np.all(o.cut_phase[-1][o.cut_iface == 1] == 1)
    assert np.all(o.cut_phase[+1][o.cut_iface == 1] == 2)
    o.assemble()
    Cs = np.zeros((6, 6))
    for k in range(6):
        u, info = o.pcg(np.eye(6)[k], tol=1e-12, green="fft")
        assert info["converged"]
        Cs[:, k] = o.mean_stress(u, np.eye(6)[k])
    Cref = _laminate_closed_form(normal, None, None, None,
                                 layers=[(fr[0], ph[0]), (fr[1], ph[1]), (fr[2], ph[2])])
    assert np.abs(Cs - Cref).max() < 1e-10 * np.abs(Cref).max()


def _hashin_bulk(N):
    Ls, ph, ell = synth.hashin_neutral_inclusion(N)
    o = XFEM(Ls, (N, N, N), ell, phases=ph)
    e = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])  # eps_bar = I
    u = o.solve_direct(e)
    s = o.mean_stress(u, e)
    return o, s[:3].sum() / 9.0  # sigma = 3 K I for eps_bar = I


def test_hashin_neutral_inclusion_bulk_modulus():
    """Sec. 4.2: K_eff = K_matrix = 1 in the continuum; the X-FEM value approaches it under
    refinement, and the enriched nodes of both interfaces are 36 % of the nodes at N = 16."""
    errs = {}
    for N in (8, 12):
        o, K = _hashin_bulk(N)
        errs[N] = abs(K - synth.HASHIN["bulk_MPa"][2])
    assert errs[12] < errs[8]
    assert errs[12] < 1e-3
    Ls, ph, ell = synth.hashin_neutral_inclusion(16)
    o = XFEM(Ls, (16, 16, 16), ell, phases=ph)
    assert round(100 * o.nX / o.nFE) == 36
    # the composite-sphere formula with the table's values (rounded to six digits) is neutral
    Ki, Kc, Km = synth.HASHIN["bulk_MPa"]
    nu = synth.HASHIN["poisson"]
    Gc = 3 * Kc * (1 - 2 * nu) / (2 * (1 + nu))
    phi = (synth.HASHIN["r_inclusion_um"] / synth.HASHIN["r_coating_um"]) ** 3
    Kcs = Kc + phi * (Ki - Kc) / (1 + (1 - phi) * (Ki - Kc) / (Kc + 4 * Gc / 3))
    assert abs(Kcs - Km) < 1e-6


def test_positive_second_levelset_is_one_interface():
    """L_1 > 0 everywhere: phase 1 never occurs and the system is the one-interface system of
    (phase 0, phase 2)."""
    n = (6, 7, 5)
    L = synth.sphere_levelset(n, (0.4, 0.55, 0.5), 0.3)
    ph = [synth.lame_from_E_nu(5.0, 0.2), synth.lame_from_E_nu(2.0, 0.3),
          synth.lame_from_E_nu(1.0, 0.35)]
    o2 = XFEM(np.stack([L, np.ones(n)]), n, phases=ph)
    o1 = XFEM(L, n, lame_minus=ph[0], lame_plus=ph[2])
    A2, S2, C2 = o2.assemble()
    A1, S1, C1 = o1.assemble()
    assert abs(A2 - A1).max() == 0.0 and abs(S2 - S1).max() == 0.0
    assert np.array_equal(C2, C1)
    assert o2.nX == o1.nX and np.array_equal(o2.D, o1.D)


def test_two_interfaces_in_one_element_refused():
    """Two concentric spheres closer than a tet: the coating is thinner than one element."""
    n = (8, 8, 8)
    c = (0.5, 0.5, 0.5)
    Ls = synth.coated_sphere_levelsets(n, c, 0.25, 0.25 + 0.3 / 8)
    ph = [(1.0, 1.0), (2.0, 2.0), (3.0, 3.0)]
    with pytest.raises(ValueError, match="two interfaces"):
        XFEM(Ls, n, phases=ph)


def test_three_phase_gradient_matches_finite_differences():
    """The envelope identity per phase (all six Lame constants and the voxel scale): central
    differences of the energy-form C_eff, and Euler homogeneity of degree one."""
    n = (10, 10, 10)
    Ls = synth.coated_sphere_levelsets(n, (0.45, 0.5, 0.55), 0.18, 0.4)
    ph = [synth.lame_from_E_nu(8.0, 0.2), synth.lame_from_E_nu(0.5, 0.35), synth.lame_from_E_nu(1.0, 0.3)]
    s = synth.voxel_scale(n, 5)

    def ceff(phases, scale):
        o = XFEM(Ls, n, phases=phases, scale=scale)
        return o, o.effective_stiffness()

    o, (Cs, Ce, U) = ceff(ph, s)
    assert set(np.unique(o.cut_iface)) == {0, 1}
    dl, ds = o.stiffness_gradient(U)
    theta = [x for p in ph for x in p]
    assert np.allclose(sum(t * g for t, g in zip(theta, dl)), Ce, atol=1e-12 * np.abs(Ce).max())
    assert np.allclose(np.einsum("v,vkl->kl", s.ravel().astype(float), ds), Ce,
                       atol=1e-12 * np.abs(Ce).max())
    for p in (1, 2, 3, 4):  # mu_0, lambda_1, mu_1, lambda_2
        hp = 1e-6 * theta[p]
        tp, tm = list(theta), list(theta)
        tp[p] += hp
        tm[p] -= hp
        _, (_, Cp, _) = ceff([tuple(tp[2 * q:2 * q + 2]) for q in range(3)], s)
        _, (_, Cm, _) = ceff([tuple(tm[2 * q:2 * q + 2]) for q in range(3)], s)
        fd = (Cp - Cm) / (2 * hp)
        assert np.abs(fd - dl[p]).max() < 1e-6 * np.abs(dl[p]).max(), p


def test_three_phase_voxel_stress_averages_to_mean_stress():
    """The per-voxel average stresses of a three-phase solution average (voxel volumes over the
    cell volume) to the mean stress, and in a voxel of one uncut phase the stress is that
    phase's C (eps_bar + grad^s u) on each tet."""
    n = (10, 10, 10)
    Ls = synth.coated_sphere_levelsets(n, (0.45, 0.5, 0.55), 0.18, 0.4)
    ph = [synth.lame_from_E_nu(8.0, 0.2), synth.lame_from_E_nu(0.5, 0.35), synth.lame_from_E_nu(1.0, 0.3)]
    o = XFEM(Ls, n, phases=ph)
    e = np.array([0.3, -0.1, 0.2, 0.4, 0.0, -0.2])
    u = o.solve_direct(e)
    vs = o.voxel_stress(u, e)
    assert np.allclose(vs.mean(axis=0), o.mean_stress(u, e), atol=1e-12 * np.abs(vs).max())
    # every phase occurs in uncut voxels; there the average stress is C_p applied to the
    # average strain of the voxel's six tets
    full = ~o.cut.any(axis=1)
    for p in range(3):
        vox = np.flatnonzero(full & (o.tet_phase == p).all(axis=1))
        assert vox.size > 0, p
        strain = e + sum(o._strains_uncut(u[None], t, vox)[0] for t in range(6)) / 6.0
        assert np.allclose(vs[vox], strain @ iso_stiffness(*ph[p]).T, atol=1e-12 * np.abs(vs).max())
