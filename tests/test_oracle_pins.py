"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: closed forms (laminate,
homogeneous cell, barycentric integrals), exact inequalities (Voigt/Reuss), invariances
(symmetry, axis permutations, translations), independent solution routes (sparse direct,
dense eigen-analysis, PCG with two different Green's operators) and a number the paper prints
(the DOF overhead of Hashin's inclusion at N = 16).
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import XFEM, classify, clip_tet, iso_stiffness, quad4, symgrad_operator

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_tet(rng):
    while True:
        X = rng.normal(size=(4, 3))
        vol = abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]]))) / 6
        if vol > 0.05:
            return X, vol


def _mandel(E):
    s2 = math.sqrt(2.0)
    return np.array([E[0, 0], E[1, 1], E[2, 2], s2 * E[1, 2], s2 * E[0, 2], s2 * E[0, 1]])


def _unmandel(v):
    s2 = math.sqrt(2.0)
    return np.array([[v[0], v[5] / s2, v[4] / s2],
                     [v[5] / s2, v[1], v[3] / s2],
                     [v[4] / s2, v[3] / s2, v[2]]])


def _bary_samples(rng, m):
    return rng.dirichlet(np.ones(4), size=m)


# --------------------------------------------------------------------------- quadrature
def test_quad4_integrates_quadratics_exactly():
    """Closed form: int_T l_i l_j = |T| (1 + delta_ij) / 20, int_T l_i = |T| / 4."""
    rng = np.random.default_rng(0)
    X, vol = _rand_tet(rng)
    bary, w = quad4()
    assert np.isclose(w.sum(), 1.0)
    for i in range(4):
        assert np.isclose(vol * np.sum(w * bary[:, i]), vol / 4, rtol=1e-14)
        for j in range(4):
            exact = vol * (2.0 if i == j else 1.0) / 20.0
            assert np.isclose(vol * np.sum(w * bary[:, i] * bary[:, j]), exact, rtol=1e-13)
    # it is a genuine degree-2 rule: the cubic l_0^3 is not integrated exactly
    assert not np.isclose(np.sum(w * bary[:, 0] ** 3), 6.0 / 120.0 * 6.0, rtol=1e-3)


# --------------------------------------------------------------------------- sub-tetrahedra
@pytest.mark.parametrize("pattern", [
    (-1, 1, 1, 1), (1, -1, 1, 1), (-1, -1, 1, 1), (1, -1, -1, 1), (-1, 1, -1, -1),
    (-1, 0, 1, 1), (-1, 0, 0, 1), (0, -1, 1, 1), (-1, -1, 0, 1), (1, 0, -1, 0)])
def test_clip_volumes_and_moments(pattern):
    rng = np.random.default_rng(abs(hash(pattern)) % 2 ** 31)
    X, vol = _rand_tet(rng)
    L = np.array(pattern, float) * rng.uniform(0.2, 1.0, size=4)
    neg = clip_tet(X, L, -1)
    pos = clip_tet(X, L, +1)
    vneg = sum(abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6 for P in neg)
    vpos = sum(abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6 for P in pos)
    assert np.isclose(vneg + vpos, vol, rtol=1e-12)
    # closed form when one vertex is alone on its side: |T| * prod of crossing fractions
    for s in (-1, 1):
        alone = [a for a in range(4) if s * L[a] > 0]
        others = [b for b in range(4) if s * L[b] < 0]
        if len(alone) == 1:
            a = alone[0]
            frac = 1.0
            for b in range(4):
                if b != a:
                    frac *= L[a] / (L[a] - L[b]) if b in others else 1.0
            vs = vneg if s < 0 else vpos
            assert np.isclose(vs, vol * frac, rtol=1e-12)
    # Monte Carlo check of the second moments int_{L<0} l_i l_j
    m = 400000
    lam = _bary_samples(rng, m)
    inside = lam @ L < 0
    mc = vol * (lam[inside].T @ lam[inside]) / m
    bary, w = quad4()
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
    Jinv = np.linalg.inv(J)
    q = np.zeros((4, 4))
    for P in neg:
        v = abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6
        pts = bary @ P
        l13 = (pts - X[0]) @ Jinv
        lb = np.concatenate([1 - l13.sum(1, keepdims=True), l13], 1)
        q += v * (lb * w[:, None]).T @ lb
    assert np.allclose(q, mc, atol=8e-3 * np.abs(mc).max())
    # exact second moments of the lone-vertex corner tet: for a tet with barycentric vertex
    # coordinates beta_v, int l_i l_j = |T'| / 20 (sum_v beta_vi beta_vj + sum_v beta_vi sum_v beta_vj)
    alone = [a for a in range(4) if L[a] < 0]
    if len(alone) == 1 and all(L[b] > 0 for b in range(4) if b != alone[0]):
        a = alone[0]
        beta = [np.eye(4)[a]]
        for b in range(4):
            if b != a:
                t = L[a] / (L[a] - L[b])
                beta.append((1 - t) * np.eye(4)[a] + t * np.eye(4)[b])
        beta = np.array(beta)
        vsub = vol * abs(np.linalg.det(beta[1:, [c for c in range(4) if c != a]] - beta[0, [c for c in range(4) if c != a]]))
        exact = vsub / 20 * (beta.T @ beta + np.outer(beta.sum(0), beta.sum(0)))
        assert np.allclose(q, exact, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------- strain operator
def test_symgrad_of_affine_field_is_exact():
    rng = np.random.default_rng(1)
    X, vol = _rand_tet(rng)
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
    G = np.zeros((4, 3))
    G[1:] = np.linalg.inv(J).T
    G[0] = -G[1:].sum(0)
    H = rng.normal(size=(3, 3))
    u = (X @ H.T).ravel()  # u_a = H X_a, node-major
    B = symgrad_operator(G)
    eps = B @ u
    assert np.allclose(eps, _mandel(0.5 * (H + H.T)), atol=1e-13)
    # Mandel inner product = tensor contraction
    S = rng.normal(size=(3, 3))
    S = S + S.T
    E = 0.5 * (H + H.T)
    assert np.isclose(_mandel(S) @ _mandel(E), np.sum(S * E))
    # iso stiffness in Mandel = lam tr(E) I + 2 mu E
    C = iso_stiffness(2.0, 3.0)
    assert np.allclose(_unmandel(C @ _mandel(E)), 2.0 * np.trace(E) * np.eye(3) + 6.0 * E)


# --------------------------------------------------------------------------- closed forms
def test_homogeneous_cell_reproduces_C():
    n = (6, 6, 6)
    lp = synth.lame_from_E_nu(2.0, 0.3)
    o = XFEM(np.ones(n), n, lame_minus=(5.0, 1.0), lame_plus=lp)
    assert o.nX == 0
    Cs, Ce, U = o.effective_stiffness()
    assert np.abs(U).max() < 1e-12
    assert np.allclose(Cs, iso_stiffness(*lp), rtol=0, atol=1e-13)
    assert np.allclose(Ce, iso_stiffness(*lp), rtol=0, atol=1e-13)


def test_equal_phases_with_cut_give_zero_fluctuation():
    n = (8, 8, 8)
    lam = synth.lame_from_E_nu(3.0, 0.25)
    L = synth.sphere_levelset(n, (0.43, 0.51, 0.47), 0.27)
    o = XFEM(L, n, lame_minus=lam, lame_plus=lam)
    assert o.nX > 0
    Cs, Ce, U = o.effective_stiffness()
    assert np.abs(U).max() < 1e-11
    assert np.allclose(Cs, iso_stiffness(*lam), atol=1e-12)


def _laminate_closed_form(normal, fraction, lm, lp, layers=None):
    """Effective stiffness of a laminate (Mandel 6x6): continuity of traction and of the
    in-plane strain; jump a_p along the normal in each layer.  Two phases (volume fraction of
    ``lm``), or ``layers`` = [(fraction, (lambda, mu)), ...]."""
    nrm = np.asarray(normal, float) / np.linalg.norm(normal)
    d = np.eye(3)

    def C4(lam, mu):
        return (lam * np.einsum("ij,kl->ijkl", d, d)
                + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))

    if layers is None:
        layers = [(fraction, lm), (1.0 - fraction, lp)]
    phases = [(f, C4(*lame)) for f, lame in layers]
    out = np.zeros((6, 6))
    for k in range(6):
        E = _unmandel(np.eye(6)[k])
        Ks = [np.einsum("j,ijkl,l->ik", nrm, C, nrm) for _, C in phases]
        lhs = sum(f * np.linalg.inv(K) for (f, _), K in zip(phases, Ks))
        rhs = sum(f * np.linalg.inv(K) @ np.einsum("ijkl,kl,j->i", C, E, nrm)
                  for (f, C), K in zip(phases, Ks))
        t = np.linalg.solve(lhs, rhs)
        sig = np.zeros((3, 3))
        for (f, C), K in zip(phases, Ks):
            a = np.linalg.solve(K, t - np.einsum("ijkl,kl,j->i", C, E, nrm))
            eps = E + 0.5 * (np.outer(a, nrm) + np.outer(nrm, a))
            sig += f * np.einsum("ijkl,kl->ij", C, eps)
        out[:, k] = _mandel(sig)
    return out


def test_tilted_laminate_matches_closed_form():
    """The laminate's exact solution (affine plus a kink along the interfaces) lies in the
    X-FEM space whenever every cut tet sees a single flat interface, so C_eff equals the
    closed-form laminate stiffness up to the solver tolerance."""
    n = (20, 20, 20)
    normal = (1, 1, 2)
    L = synth.laminate_levelset(n, normal=normal, offset=0.137, fraction=0.5)
    lm = synth.lame_from_E_nu(10.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    # the premise: inside every cut tet the nodal level set is one affine function
    m = np.asarray(normal, float) / np.linalg.norm(normal)
    for v, t in o.cut_list[:: max(1, len(o.cut_list) // 400)]:
        X = (o.vox_ijk[v] + o.tet_offsets[t]) * o.h
        Lv = o.L[o.tet_nodes[v, t]]
        c = Lv - X @ m
        assert np.ptp(c) < 1e-12 or np.ptp(Lv + X @ m) < 1e-12
    Cref = _laminate_closed_form(normal, 0.5, lm, lp)
    o.assemble()
    Cs = np.zeros((6, 6))
    for k in range(6):
        u, info = o.pcg(np.eye(6)[k], tol=1e-12, green="fft")
        assert info["converged"]
        Cs[:, k] = o.mean_stress(u, np.eye(6)[k])
    assert np.abs(Cs - Cref).max() < 1e-9 * np.abs(Cref).max()


# --------------------------------------------------------------------------- bounds, symmetry
@pytest.fixture(scope="module")
def sphere10():
    n = (10, 10, 10)
    L = synth.sphere_levelset(n, (0.5, 0.5, 0.5), 0.3)
    lm = synth.lame_from_E_nu(10.0, 0.3)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    Cs, Ce, U = o.effective_stiffness()
    return o, Cs, Ce, U, lm, lp


def test_symmetry_and_axis_permutation_invariance(sphere10):
    o, Cs, Ce, U, lm, lp = sphere10
    assert np.abs(Ce - Ce.T).max() < 1e-13 * np.abs(Ce).max()
    assert np.abs(Cs - Ce).max() < 1e-10 * np.abs(Ce).max()
    sc = np.abs(Ce).max()
    for a, b in [(0, 1), (0, 2)]:
        assert abs(Ce[a, a] - Ce[b, b]) < 1e-12 * sc
    for a, b in [(3, 4), (3, 5)]:
        assert abs(Ce[a, a] - Ce[b, b]) < 1e-12 * sc
    assert abs(Ce[0, 1] - Ce[0, 2]) < 1e-12 * sc and abs(Ce[0, 1] - Ce[1, 2]) < 1e-12 * sc


def test_voigt_reuss_bounds(sphere10):
    """u = 0 is admissible (Voigt) and V_h is a subspace of H^1 (Reuss), with the phase
    volumes of the linearised interface."""
    o, Cs, Ce, U, lm, lp = sphere10
    vol = {-1: 0.0, 1: 0.0}
    for t in range(6):
        ph = o.tet_phase[~o.cut[:, t], t]  # phase index: 0 minus, 1 plus
        for s in (-1, 1):
            vol[s] += o.tet_vol[t] * np.sum(ph == (s + 1) // 2)
    for idx in range(len(o.cut_list)):
        _, sides = o.cut_data[idx]
        for s in (-1, 1):
            vol[s] += sides[s][1].sum()
    f = {s: vol[s] / o.volY for s in vol}
    assert np.isclose(f[-1] + f[1], 1.0)
    C = {-1: iso_stiffness(*lm), 1: iso_stiffness(*lp)}
    voigt = f[-1] * C[-1] + f[1] * C[1]
    reuss = np.linalg.inv(f[-1] * np.linalg.inv(C[-1]) + f[1] * np.linalg.inv(C[1]))
    assert np.linalg.eigvalsh(voigt - Ce).min() > -1e-12
    assert np.linalg.eigvalsh(Ce - reuss).min() > -1e-12
    assert np.linalg.eigvalsh(voigt - Ce).max() > 1e-3  # not trivially at a bound
    # Hashin-Shtrikman bounds on the bulk modulus of the isotropic projection (soft check)
    Kp = [lam + 2 * mu / 3 for lam, mu in (lm, lp)]
    Gp = [mu for lam, mu in (lm, lp)]
    K_eff = np.sum(Ce[:3, :3]) / 9.0
    fi, fm = f[-1], f[1]
    Ki, Km, Gi, Gm = Kp[0], Kp[1], Gp[0], Gp[1]
    hs_lo = Km + fi / (1 / (Ki - Km) + 3 * fm / (3 * Km + 4 * Gm))
    hs_hi = Ki + fm / (1 / (Km - Ki) + 3 * fi / (3 * Ki + 4 * Gi))
    assert hs_lo * 0.98 <= K_eff <= hs_hi * 1.02


def test_pcg_matches_direct_on_ragged_grid():
    n = (10, 12, 8)
    L = np.minimum(synth.sphere_levelset(n, (0.3, 0.4, 0.5), 0.22),
                   synth.sphere_levelset(n, (0.8, 0.85, 0.2), 0.15))
    o = XFEM(L, n, lame_minus=synth.lame_from_E_nu(20.0, 0.2), lame_plus=synth.lame_from_E_nu(1.0, 0.3))
    e = np.array([0.3, -0.1, 0.2, 0.05, 0.1, -0.2])
    ud = o.solve_direct(e)
    for green in ("sparse", "fft"):
        up, info = o.pcg(e, tol=1e-12, green=green)
        assert info["converged"]
        assert np.abs(up - ud).max() < 1e-9 * np.abs(ud).max()
    # the direct solution solves the system with a mean-free standard part
    r = o.A @ ud + o.rhs(e)
    assert np.abs(r).max() < 1e-11 * np.abs(o.rhs(e)).max()
    assert np.abs(ud[: 3 * o.nFE].reshape(3, -1).sum(1)).max() < 1e-12


def test_dense_bruteforce_tiny_grid():
    """N = 3: the dense matrix has exactly the three standard translations as kernel."""
    n = (3, 3, 3)
    L = synth.sphere_levelset(n, (0.5, 0.5, 0.5), 0.3)
    o = XFEM(L, n, lame_minus=synth.lame_from_E_nu(5.0, 0.3), lame_plus=synth.lame_from_E_nu(1.0, 0.3))
    assert o.nX > 0
    A, _, _ = o.assemble()
    Ad = A.toarray()
    w, V = np.linalg.eigh(Ad)
    assert np.sum(np.abs(w) < 1e-10 * w.max()) == 3 and w.min() > -1e-10 * w.max()
    null = V[:, :3]
    T = np.zeros((o.ndof, 3))
    for c in range(3):
        T[c * o.nFE:(c + 1) * o.nFE, c] = 1.0
    assert np.allclose(null @ (null.T @ T), T, atol=1e-10)
    e = np.eye(6)[3]
    u = o.solve_direct(e)
    upinv = -np.linalg.pinv(Ad, rcond=1e-12) @ o.rhs(e)
    assert np.allclose(u, upinv, atol=1e-10 * np.abs(u).max())


def test_green_symbol_equals_assembled_reference_operator():
    n = (6, 8, 10)
    o = XFEM(np.ones(n), n)
    A0 = o.assemble_reference()
    rng = np.random.default_rng(3)
    u = rng.normal(size=3 * o.nFE)
    M = o.green_symbol()
    U = np.fft.fftn(u.reshape((3,) + n), axes=(1, 2, 3))
    Au = np.real(np.fft.ifftn(np.einsum("...ij,j...->i...", M, U), axes=(1, 2, 3))).ravel()
    assert np.allclose(Au, A0 @ u, atol=1e-12 * np.abs(A0 @ u).max())
    # Hermitian, positive definite away from xi = 0
    assert np.allclose(M, np.conj(np.swapaxes(M, -1, -2)))
    ev = np.linalg.eigvalsh(M.reshape(-1, 3, 3)[1:])
    assert ev.min() > 0
    f = A0 @ u
    zs = o.precondition(np.concatenate([f, np.zeros(0)]), green="sparse")
    zf = o.precondition(np.concatenate([f, np.zeros(0)]), green="fft")
    ref = u.reshape(3, -1) - u.reshape(3, -1).mean(1, keepdims=True)
    assert np.allclose(zs, ref.ravel(), atol=1e-9)
    assert np.allclose(zf, ref.ravel(), atol=1e-9)


def test_single_mode_green_symbol_and_plane_waves():
    """green_symbol_at equals the full symbol array (itself pinned to the assembled reference
    operator above) on a ragged anisotropic grid, and the plane-wave preconditioner equals the
    FFT preconditioner on a superposition of modes that includes Nyquist and zero components."""
    n = (4, 6, 8)
    o = XFEM(np.ones(n), n, (1.3, 0.7, 1.1))
    M = o.green_symbol()
    rng = np.random.default_rng(3)
    for kv in [(0, 0, 1), (2, 3, 4), (1, 5, 7), (3, 0, 4), (2, 3, 0)]:
        assert np.allclose(o.green_symbol_at(kv), M[kv], rtol=1e-13, atol=1e-13)
    modes = [((k0, k1, k2), rng.normal(size=3) + 1j * rng.normal(size=3))
             for (k0, k1, k2) in [(0, 0, 4), (2, 3, 0), (1, 2, 3), (0, 3, 4), (3, 5, 1), (2, 0, 0)]]
    f, z = o.precondition_modes(modes)
    zf = o.precondition(f, green="fft")
    assert np.allclose(z, zf, rtol=1e-11, atol=1e-11 * np.abs(zf).max())


def test_enriched_block_preconditioner():
    """Variant enriched preconditioner (3x3 node blocks): each block equals the node block of the
    scaled stiffness assembled with C = I_sym (lambda = 0, mu = 1/2), an independent route through
    the element integration; the blocks have unit diagonal (the per-DOF scaling) and are SPD; PCG
    with them reaches the direct solution (the preconditioner does not change the system)."""
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    o = XFEM(L, n, lame_minus=(0.0, 0.5), lame_plus=(0.0, 0.5))
    o.assemble()
    n3 = 3 * o.nFE
    A = o.A.tocsr()
    for j in range(0, o.nX, max(1, o.nX // 25)):
        idx = [n3 + c * o.nX + j for c in range(3)]
        blk = A[idx][:, idx].toarray()
        assert np.allclose(blk, o.Bblk[j], rtol=1e-12, atol=1e-12)
    assert np.allclose(np.einsum("jkk->jk", o.Bblk), 1.0, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(o.Bblk) > 0.0)
    o2 = XFEM(L, n, lame_minus=synth.lame_from_E_nu(1.0, 0.3), lame_plus=synth.lame_from_E_nu(10.0, 0.3))
    e = np.eye(6)[3]
    ud = o2.solve_direct(e)
    ub, info_b = o2.pcg(e, tol=1e-12, enr="block3")
    ui, info_i = o2.pcg(e, tol=1e-12)
    assert np.linalg.norm(ub - ud) < 1e-9 * np.linalg.norm(ud)
    assert np.linalg.norm(ui - ud) < 1e-9 * np.linalg.norm(ud)


def test_basic_and_barzilai_borwein_schemes():
    """The basic scheme (Richardson with s0 = 2/(C_- + C_+), eq. stepsize), Barzilai-Borwein and
    nonlinear CG on the same X-FFT system reach the direct solution; the basic scheme's iteration
    count grows about linearly with the contrast and much faster than linear CG's (Sec. 2.3's
    remarks on O(kappa) and O(sqrt kappa)); BB needs far fewer iterations than the basic scheme;
    nonlinear CG needs more than linear CG but at most twice as many (Sec. 2.3)."""
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    e = np.eye(6)[0]
    its = {}
    for contrast in (10.0, 50.0):
        o = XFEM(L, n, lame_minus=synth.lame_from_E_nu(contrast, 0.2), lame_plus=synth.lame_from_E_nu(1.0, 0.3))
        ud = o.solve_direct(e)
        lam, mu = o.phases[0]
        assert math.isclose(o.basic_step(), 2.0 / (2 * o.phases[1][1] + 3 * lam + 2 * mu), rel_tol=1e-15)
        for scheme in ("cg", "basic", "bb", "nlcg"):
            u, info = o.pcg(e, tol=1e-10, maxit=5000, scheme=scheme)
            assert info["converged"], (contrast, scheme)
            assert np.linalg.norm(u - ud) < 1e-8 * np.linalg.norm(ud)
            its[scheme, contrast] = info["iters"]
    assert its["basic", 50.0] > 3.0 * its["basic", 10.0]
    assert its["basic", 50.0] / its["basic", 10.0] > 1.5 * its["cg", 50.0] / its["cg", 10.0]
    for c in (10.0, 50.0):
        assert its["bb", c] < 0.5 * its["basic", c]
        assert its["cg", c] <= its["bb", c]
        assert its["cg", c] < its["nlcg", c] <= 2 * its["cg", c]


def test_extreme_contrasts_with_both_enriched_preconditioners():
    """Contrast 1e-4 (nearly a pore) and 1e4 (nearly rigid): PCG with the identity and with the
    block enriched preconditioner both reach the direct solution (the preconditioner changes
    the iteration count only)."""
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    e = np.eye(6)[0]
    for contrast in (1e-4, 1e4):
        o = XFEM(L, n, lame_minus=synth.lame_from_E_nu(contrast, 0.3), lame_plus=synth.lame_from_E_nu(1.0, 0.3))
        ud = o.solve_direct(e)
        for enr in ("identity", "block3"):
            u, info = o.pcg(e, tol=1e-10, maxit=5000, enr=enr)
            assert info["converged"], (contrast, enr)
            assert np.linalg.norm(u - ud) < 1e-6 * np.linalg.norm(ud), (contrast, enr)


def test_hashin_dof_overhead_matches_paper():
    """Sec. 4.2: 36% more DOFs at N = 16 for the coated sphere (both interfaces enriched)."""
    g = json.load(open(os.path.join(HERE, "golden", "hashin_neutral_inclusion.json")))
    N = 16
    ell = (g["cell_edge_um"],) * 3
    n = (N, N, N)
    c = tuple(x / 2 for x in ell)
    L1 = synth.sphere_levelset(n, c, 6 * math.e / 5, ell)
    L2 = synth.sphere_levelset(n, c, 2 * math.pi, ell)
    tau = 1e-6 * ell[0] / N
    _, J1 = classify(L1, n, tau)
    _, J2 = classify(L2, n, tau)
    ratio = np.union1d(J1, J2).size / N ** 3
    assert round(100 * ratio) == g["dof_overhead_percent_at_N16"]
    # and the composite-sphere formula confirms the neutral-inclusion parameters
    Km, Kc, Ki = (g["bulk_modulus_MPa"][k] for k in ("matrix", "coating", "inclusion"))
    nu = g["poisson"]
    Gc = 3 * Kc * (1 - 2 * nu) / (2 * (1 + nu))
    phi = (6 * math.e / 5) ** 3 / (2 * math.pi) ** 3
    Keff = Kc + phi * (Ki - Kc) / (1 + (1 - phi) * (Ki - Kc) / (Kc + 4 * Gc / 3))
    assert abs(Keff - Km) < 1e-6


def test_translation_by_whole_nodes():
    n = (8, 10, 6)
    L = synth.sphere_levelset(n, (0.37, 0.52, 0.61), 0.28)
    lm = synth.lame_from_E_nu(7.0, 0.25)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    shift = (3, -2, 1)
    o1 = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    o2 = XFEM(np.roll(L, shift, axis=(0, 1, 2)), n, lame_minus=lm, lame_plus=lp)
    e = np.eye(6)[4]
    u1 = o1.solve_direct(e)
    u2 = o2.solve_direct(e)
    s1 = o1.mean_stress(u1, e)
    s2 = o2.mean_stress(u2, e)
    assert np.allclose(s1, s2, atol=1e-12)
    std1 = u1[: 3 * o1.nFE].reshape((3,) + n)
    std2 = u2[: 3 * o2.nFE].reshape((3,) + n)
    assert np.allclose(np.roll(std1, shift, axis=(1, 2, 3)), std2, atol=1e-11)


# --------------------------------------------------------------------------- gradient
@pytest.fixture(scope="module")
def grad_case():
    n = (6, 6, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    lm = synth.lame_from_E_nu(8.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    s = synth.voxel_scale(n, 7)
    return n, L, lm, lp, s


def _ceff(n, L, lm, lp, s):
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp, scale=s)
    return o, o.effective_stiffness()


def test_gradient_matches_finite_differences_and_euler(grad_case):
    n, L, lm, lp, s = grad_case
    o, (Cs, Ce, U) = _ceff(n, L, lm, lp, s)
    dl, ds = o.stiffness_gradient(U)
    theta = [lm[0], lm[1], lp[0], lp[1]]
    # Euler: C_eff is homogeneous of degree one in the moduli and in the scale field
    assert np.allclose(sum(t * g for t, g in zip(theta, dl)), Ce, atol=1e-12 * np.abs(Ce).max())
    assert np.allclose(np.einsum("v,vkl->kl", s.ravel().astype(float), ds), Ce,
                       atol=1e-12 * np.abs(Ce).max())
    # central differences on the energy form (quadratically accurate in the solver error)
    for p in range(4):
        hp = 1e-6 * theta[p]
        th_p = list(theta)
        th_m = list(theta)
        th_p[p] += hp
        th_m[p] -= hp
        _, (_, Cp, _) = _ceff(n, L, (th_p[0], th_p[1]), (th_p[2], th_p[3]), s)
        _, (_, Cm, _) = _ceff(n, L, (th_m[0], th_m[1]), (th_m[2], th_m[3]), s)
        fd = (Cp - Cm) / (2 * hp)
        assert np.abs(fd - dl[p]).max() < 1e-6 * np.abs(dl[p]).max()
    rng = np.random.default_rng(11)
    dirn = rng.normal(size=s.size)
    hs = 1e-6
    sp_ = s.ravel().astype(float) + hs * dirn
    sm_ = s.ravel().astype(float) - hs * dirn
    _, (_, Cp, _) = _ceff(n, L, lm, lp, sp_.reshape(n))
    _, (_, Cm, _) = _ceff(n, L, lm, lp, sm_.reshape(n))
    fd = (Cp - Cm) / (2 * hs)
    an = np.einsum("v,vkl->kl", dirn, ds)
    assert np.abs(fd - an).max() < 1e-6 * np.abs(an).max()


@pytest.mark.parametrize("normal", [(1, 0, 1), (1, 0, 0)])
def test_interfaces_through_nodes(normal):
    """Degenerate cut geometry: laminate planes through node lines (normal (1,0,1)) or node
    planes (normal (1,0,0)) at offset 1/4 on an 8^3 grid.  The snapped zero vertices put every
    cut tet's interface through a vertex (the clip's degenerate cases), and a tet that touches
    the interface only at zero vertices is not cut (with node planes no tet is cut and nothing is
    enriched); the closed form still holds to rounding."""
    n = (8, 8, 8)
    L = synth.laminate_levelset(n, normal=normal, offset=0.25, fraction=0.5)
    lm = synth.lame_from_E_nu(10.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    assert (o.L == 0.0).sum() == 128
    if normal == (1, 0, 0):
        assert len(o.cut_list) == 0 and o.nX == 0
    else:
        Lt = o.L[o.tet_nodes[o.cut]]
        assert len(o.cut_list) > 0 and np.all((Lt == 0.0).any(axis=1))
    o.assemble()
    C = np.zeros((6, 6))
    for k in range(6):
        e = np.eye(6)[k]
        C[:, k] = o.mean_stress(o.solve_direct(e), e)
    Cref = _laminate_closed_form(normal, 0.5, lm, lp)
    assert np.abs(C - Cref).max() < 1e-12 * np.abs(Cref).max()
