"""GPU <-> oracle parity through the C-ABI (libxfft.so).

Every comparison uses the same seeded inputs on both sides.  Tolerances: the FP64 path must
match the oracle's effective stiffness to relative 1e-10 and fields to relative L2 1e-9; the
FP32 kernels (single apply / preconditioner) to relative 1e-5 of the vector norm, and the
FP32-refined solve to relative 1e-6 in C_eff.  Integer setup results (classification, enriched
numbering) are bit-exact.
"""
import math

import numpy as np
import pytest

import synth
from oracle import XFEM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_02172_gb300 as pkg
    return pkg


def _case(name):
    if name == "sphere16":
        n = (16, 16, 16)
        L = synth.sphere_levelset(n, (0.5, 0.5, 0.5), 0.3)
        return n, (1.0, 1.0, 1.0), L, synth.lame_from_E_nu(10.0, 0.3), synth.lame_from_E_nu(1.0, 0.3), None
    if name == "ragged":
        n = (10, 12, 8)
        L = np.minimum(synth.sphere_levelset(n, (0.3, 0.4, 0.5), 0.22),
                       synth.sphere_levelset(n, (0.8, 0.85, 0.2), 0.15))
        return (n, (1.0, 1.0, 1.0), L, synth.lame_from_E_nu(20.0, 0.2), synth.lame_from_E_nu(1.0, 0.3),
                synth.voxel_scale(n, 3))
    if name == "fast_mixed":  # every axis on the compile-time FFT plans, radices 2, 3, 4, 8
        n = (16, 48, 32)
        L = synth.sphere_levelset(n, (0.4, 0.55, 0.5), 0.28)
        return n, (1.0, 1.2, 0.9), L, synth.lame_from_E_nu(30.0, 0.2), synth.lame_from_E_nu(1.0, 0.3), None
    if name == "fast_radix5":
        n = (80, 16, 16)
        L = synth.sphere_levelset(n, (0.5, 0.5, 0.5), 0.3)
        return n, (1.0, 1.0, 1.0), L, synth.lame_from_E_nu(5.0, 0.3), synth.lame_from_E_nu(1.0, 0.3), None
    if name == "aniso_cell":
        n = (12, 8, 10)
        ell = (1.5, 0.8, 1.2)
        L = synth.sphere_levelset(n, (0.7, 0.35, 0.6), 0.3, ell)
        return n, ell, L, synth.lame_from_E_nu(0.1, 0.35), synth.lame_from_E_nu(1.0, 0.3), None
    if name == "tiles":  # several x chunks, y and z tiles with ragged last tiles, cubic voxels
        n = (96, 48, 32)
        ell = (1.0, 0.5, 1.0 / 3.0)
        L = np.minimum(synth.sphere_levelset(n, (0.3, 0.2, 0.15), 0.11, ell),
                       synth.sphere_levelset(n, (0.75, 0.4, 0.25), 0.09, ell))
        return n, ell, L, synth.lame_from_E_nu(30.0, 0.2), synth.lame_from_E_nu(1.0, 0.3), synth.voxel_scale(n, 7)
    raise KeyError(name)


_ORACLES = {}


def _oracle(name):
    """The oracle of case `name`, built once per test module (its assembly and LU factorisation
    are cached on the object, so later tests reuse them)."""
    if name not in _ORACLES:
        n, ell, L, lm, lp, sc = _case(name)
        _ORACLES[name] = XFEM(L, n, ell, lame_minus=lm, lame_plus=lp, scale=sc)
    return _ORACLES[name]


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("name", ["sphere16", "ragged", "aniso_cell"])
def test_setup_matches_oracle(xf, name):
    n, ell, L, lm, lp, sc = _case(name)
    s = xf.Solver(n, ell)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle(name)
    en, D0, code = s.setup_info()
    assert s.num_enriched == o.nX
    assert s.num_cut_tets == len(o.cut_list)
    assert np.array_equal(en, o.enr_nodes)
    # tet codes: 2 = cut, else 0 / 1 = minus / plus phase
    exp = np.zeros(o.nvox, dtype=np.uint16)
    for t in range(6):
        bits = np.where(o.cut[:, t], 2, o.tet_phase[:, t]).astype(np.uint16)
        exp |= bits << (2 * t)
    assert np.array_equal(code, exp)
    assert _rel(D0, o.D) < 1e-12


@pytest.mark.parametrize("name", ["sphere16", "ragged", "aniso_cell"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "dw"])
def test_apply_matches_oracle(xf, name, prec):
    n, ell, L, lm, lp, sc = _case(name)
    s = xf.Solver(n, ell)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle(name)
    o.assemble()
    rng = np.random.default_rng(5)
    d = rng.normal(size=(2, o.ndof))
    eps = rng.normal(size=(2, 6))
    tol = {"fp64": 1e-12, "dw": 1e-11, "fp32": 2e-5}[prec]
    q, sig = s.apply(d, precision=prec)
    for r in range(2):
        assert _rel(q[r], o.A @ d[r]) < tol
    q, sig = s.apply(d, eps=eps, precision=prec)
    for r in range(2):
        assert _rel(q[r], o.A @ d[r] + o.rhs(eps[r])) < tol
        ref = np.asarray(o.Sm @ d[r]).ravel() + o.Cbar @ eps[r]
        assert _rel(sig[r], ref) < tol


@pytest.mark.parametrize("name", ["sphere16", "ragged", "aniso_cell"])
def test_cached_cut_apply_matches_oracle(xf, name):
    """The apply of the FP32 CG iterations (no stress integrals): the cut tets from the cached
    scaled element matrices (option cut_cache) and from the per-side moments (the default), both
    against the oracle's assembled operator."""
    n, ell, L, lm, lp, sc = _case(name)
    o = _oracle(name)
    o.assemble()
    d = np.random.default_rng(21).normal(size=(3, o.ndof))
    for cache in (True, False):
        s = xf.Solver(n, ell, precision="fp32", cut_cache=cache)
        s.set_microstructure(L, lm, lp, sc)
        q, sig = s.apply(d, precision="fp32", stress=False)
        assert sig is None
        for r in range(3):
            assert _rel(q[r], o.A @ d[r]) < 2e-5, (cache, r)


@pytest.mark.parametrize("normal", [(1, 0, 1), (1, 0, 0)])
def test_interfaces_through_nodes(xf, normal):
    """Degenerate cut geometry (snapped zero vertices on every cut tet, or no cut tet at all):
    setup bit-exact, apply as the oracle's, C_eff = the laminate closed form."""
    from test_oracle_pins import _laminate_closed_form
    n = (8, 8, 8)
    L = synth.laminate_levelset(n, normal=normal, offset=0.25, fraction=0.5)
    lm = synth.lame_from_E_nu(10.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    o.assemble()
    s = xf.Solver(n, tol=1e-12)
    s.set_microstructure(L, lm, lp)
    en, D0, code = s.setup_info()
    assert s.num_enriched == o.nX and s.num_cut_tets == len(o.cut_list)
    assert np.array_equal(en, o.enr_nodes)
    if o.nX:
        assert _rel(D0, o.D) < 1e-12
    d = np.random.default_rng(2).normal(size=(2, o.ndof))
    q, _ = s.apply(d, precision="fp64")
    for r in range(2):
        assert _rel(q[r], o.A @ d[r]) < 1e-12
    C, st = s.effective_stiffness()
    assert st["converged"]
    Cref = _laminate_closed_form(normal, 0.5, lm, lp)
    assert np.abs(C - Cref).max() < 1e-9 * np.abs(Cref).max()


def test_fp32_solve_with_cut_cache(xf):
    """FP32-refined C_eff with the cached cut-tet matrices in the CG iterations (graph-replayed)
    equals the default solve and the oracle's."""
    n, ell, L, lm, lp, sc = _case("ragged")
    o = _oracle("ragged")
    Cs, _, _ = o.effective_stiffness()
    out = {}
    for cache in (True, False):
        s = xf.Solver(n, ell, precision="fp32", tol=1e-8, cut_cache=cache)
        s.set_microstructure(L, lm, lp, sc)
        out[cache], st = s.effective_stiffness()
        assert st["converged"]
        assert np.abs(out[cache] - Cs).max() < 1e-6 * np.abs(Cs).max()
    assert np.abs(out[True] - out[False]).max() < 1e-6 * np.abs(Cs).max()


@pytest.mark.parametrize("name", ["sphere16", "ragged", "aniso_cell"])
def test_dw_residual_at_the_solution(xf, name):
    """At the exact solution the residual A u + b cancels to rounding: the double-word kernels
    must resolve it to far below the FP32 level (what the refinement's stopping rule needs)."""
    n, ell, L, lm, lp, sc = _case(name)
    s = xf.Solver(n, ell)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle(name)
    o.assemble()
    eps = np.eye(6)[[0, 3]]
    u = np.stack([o.solve_direct(e) for e in eps])
    bn = [np.linalg.norm(o.rhs(e)) for e in eps]
    q64, _ = s.apply(u, eps=eps, precision="fp64")
    qdw, _ = s.apply(u, eps=eps, precision="dw")
    q32, _ = s.apply(u, eps=eps, precision="fp32")
    for r in range(2):
        assert np.linalg.norm(q64[r]) < 1e-10 * bn[r]  # u solves the system
        assert np.linalg.norm(qdw[r] - q64[r]) < 1e-11 * bn[r]
        # FP32 cannot resolve it: the check above would fail for the FP32 kernels
        assert np.linalg.norm(q32[r] - q64[r]) > 1e-9 * bn[r]


@pytest.mark.parametrize("name", ["sphere16", "ragged", "aniso_cell", "fast_mixed", "fast_radix5"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_precondition_matches_oracle(xf, name, prec):
    n, ell, L, lm, lp, sc = _case(name)
    s = xf.Solver(n, ell)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle(name)
    rng = np.random.default_rng(9)
    f = rng.normal(size=(3, o.ndof))
    for r in range(3):  # the standard part must be mean-free per component
        std = f[r, : 3 * o.nFE].reshape(3, -1)
        std -= std.mean(axis=1, keepdims=True)
    z, rr = s.precondition(f, precision=prec)
    tol = 1e-11 if prec == "fp64" else 2e-5
    green = "fft" if name.startswith("fast") else "sparse"
    for r in range(3):
        ref = o.precondition(f[r], green=green)
        assert _rel(z[r], ref) < tol
        assert abs(rr[r] - f[r] @ ref) <= tol * abs(f[r] @ ref) * 10


@pytest.mark.parametrize("name", ["sphere16", "ragged", "aniso_cell"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_enriched_preconditioner(xf, name, prec):
    """Variant enriched preconditioner (3x3 node blocks): P^-1 against the oracle, and a solve
    with it reaching the direct solution (the system does not depend on the preconditioner)."""
    n, ell, L, lm, lp, sc = _case(name)
    o = _oracle(name)
    s = xf.Solver(n, ell, precision=prec, tol=1e-12 if prec == "fp64" else 1e-10, enr_precond="block3")
    s.set_microstructure(L, lm, lp, sc)
    rng = np.random.default_rng(13)
    f = rng.normal(size=(2, o.ndof))
    for r in range(2):
        std = f[r, : 3 * o.nFE].reshape(3, -1)
        std -= std.mean(axis=1, keepdims=True)
    z, rr = s.precondition(f, precision=prec)
    tol = 1e-11 if prec == "fp64" else 2e-5
    for r in range(2):
        ref = o.precondition(f[r], green="sparse", enr="block3")
        assert _rel(z[r], ref) < tol
    eps = np.array([[0.2, -0.1, 0.3, 0.4, -0.2, 0.1]])
    out = s.solve(eps, u=True)
    assert out["converged"], out["stats"]
    u = o.solve_direct(eps[0])
    ms = o.mean_stress(u, eps[0])
    ctol = 1e-10 if prec == "fp64" else 1e-6
    assert np.abs(out["mean_stress"][0] - ms).max() < ctol * np.abs(ms).max()
    if prec == "fp64":
        assert _rel(out["u_std"][0], u[: 3 * o.nFE].reshape(3, -1)) < 1e-9


@pytest.mark.parametrize("scheme", ["basic", "bb", "nlcg"])
def test_basic_and_bb_schemes(xf, scheme):
    """The basic (Richardson, step s0 of eq. stepsize), Barzilai-Borwein and nonlinear CG schemes
    on the same system: FP64 iteration counts as the oracle's (up to rounding) and the direct
    solution; the FP32-refined form reaches the same mean stress to 1e-6."""
    n, ell, L, lm, lp, sc = _case("sphere16")
    o = _oracle("sphere16")
    eps = np.array([[0.2, -0.1, 0.3, 0.4, -0.2, 0.1]])
    u_ref = o.solve_direct(eps[0])
    _, info = o.pcg(eps[0], tol=1e-10, maxit=5000, scheme=scheme, green="fft")
    s = xf.Solver(n, ell, tol=1e-10, maxit=5000, scheme=scheme)
    s.set_microstructure(L, lm, lp, sc)
    out = s.solve(eps, u=True)
    assert out["converged"], out["stats"]
    assert abs(out["stats"]["iters"][0] - info["iters"]) <= 2, (out["stats"]["iters"], info["iters"])
    assert _rel(out["u_std"][0], u_ref[: 3 * o.nFE].reshape(3, -1)) < 1e-8
    ms = o.mean_stress(u_ref, eps[0])
    s32 = xf.Solver(n, ell, precision="fp32", tol=1e-9, maxit=5000, scheme=scheme)
    s32.set_microstructure(L, lm, lp, sc)
    out32 = s32.solve(eps, u=False)
    assert out32["converged"], out32["stats"]
    assert np.abs(out32["mean_stress"][0] - ms).max() < 1e-6 * np.abs(ms).max()


def test_one_call_solve(xf):
    """The one-call Python solve equals the oracle's direct solution (sphere16)."""
    n, ell, L, lm, lp, sc = _case("sphere16")
    o = _oracle("sphere16")
    eps = np.array([[0.3, 0.1, -0.2, 0.0, 0.5, 0.0]])
    out = xf.solve(L, lm, lp, eps, precision="fp64", tol=1e-12)
    assert out["converged"]
    u = o.solve_direct(eps[0])
    assert _rel(out["u_std"][0], u[: 3 * o.nFE].reshape(3, -1)) < 1e-9


@pytest.mark.parametrize("name", ["sphere16", "ragged"])
def test_fp64_solve_matches_direct(xf, name):
    n, ell, L, lm, lp, sc = _case(name)
    s = xf.Solver(n, ell, tol=1e-12)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle(name)
    eps = np.array([[1.0, 0, 0, 0, 0, 0], [0.2, -0.1, 0.3, 0.4, -0.2, 0.1]])
    out = s.solve(eps, u=True, voxel_stress=True)
    assert out["converged"], out["stats"]
    for r in range(2):
        u = o.solve_direct(eps[r])
        ustd = u[: 3 * o.nFE].reshape(3, -1)
        uenr = (u[3 * o.nFE:].reshape(3, -1) * o.Dinvsqrt.T)
        assert _rel(out["u_std"][r], ustd) < 1e-9
        if o.nX:
            assert _rel(out["u_enr"][r], uenr) < 1e-9
        ms = o.mean_stress(u, eps[r])
        assert np.abs(out["mean_stress"][r] - ms).max() < 1e-10 * np.abs(ms).max()
        vs = o.voxel_stress(u, eps[r])
        assert _rel(out["voxel_stress"][r], vs.T) < 1e-9


def test_fp64_effective_stiffness_and_gradient(xf):
    n, ell, L, lm, lp, sc = _case("ragged")
    s = xf.Solver(n, ell, tol=1e-12)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle("ragged")
    C, st = s.effective_stiffness()
    assert st["converged"]
    Cs, Ce, U = o.effective_stiffness()
    assert np.abs(C - Cs).max() < 1e-10 * np.abs(Cs).max()
    rng = np.random.default_rng(2)
    G = rng.normal(size=(6, 6))
    dl, ds, Cenergy = s.grad(G)
    assert np.abs(Cenergy - Ce).max() < 1e-10 * np.abs(Ce).max()
    dlr, dsr = o.stiffness_gradient(U)
    ref_l = np.einsum("kl,pkl->p", G, dlr)
    ref_s = np.einsum("kl,vkl->v", G, dsr)
    assert np.abs(dl - ref_l).max() < 1e-9 * np.abs(ref_l).max()
    assert _rel(ds.astype(np.float64), ref_s) < 1e-6  # float32 output


def test_fp32_refined_effective_stiffness(xf):
    n, ell, L, lm, lp, sc = _case("ragged")
    s = xf.Solver(n, ell, precision="fp32", tol=1e-10)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle("ragged")
    C, st = s.effective_stiffness()
    assert st["converged"], st
    Cs, Ce, U = o.effective_stiffness()
    assert np.abs(C - Cs).max() < 1e-6 * np.abs(Cs).max()


def test_fp32_refined_gradient(xf):
    """Mixed-precision solver: standard strains from float-pair node differences, enriched strains
    from FP64 differences, FP32 strain products and FP64 sums stay within the accuracy of the
    tol-limited solution."""
    n, ell, L, lm, lp, sc = _case("ragged")
    s = xf.Solver(n, ell, precision="fp32", tol=1e-10)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle("ragged")
    C, st = s.effective_stiffness()
    assert st["converged"], st
    Cs, Ce, U = o.effective_stiffness()
    G = np.random.default_rng(2).normal(size=(6, 6))
    dl, ds, Cenergy = s.grad(G)
    assert np.abs(Cenergy - Ce).max() < 1e-6 * np.abs(Ce).max()
    dlr, dsr = o.stiffness_gradient(U)
    ref_l = np.einsum("kl,pkl->p", G, dlr)
    ref_s = np.einsum("kl,vkl->v", G, dsr)
    assert np.abs(dl - ref_l).max() < 1e-5 * np.abs(ref_l).max()
    assert _rel(ds.astype(np.float64), ref_s) < 1e-5


def test_gradient_against_finite_differences(xf):
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    lm = synth.lame_from_E_nu(8.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    sc = synth.voxel_scale(n, 7)
    rng = np.random.default_rng(4)
    Ct = rng.normal(size=(6, 6))

    def ceff(lmv, lpv, scv):
        s = xf.Solver(n, tol=1e-13)
        s.set_microstructure(L, lmv, lpv, scv)
        C, st = s.effective_stiffness()
        return s, C

    s, C = ceff(lm, lp, sc)
    G = 2.0 * (C - Ct)
    dl, ds, _ = s.grad(G)
    theta = [lm[0], lm[1], lp[0], lp[1]]
    for p in range(4):
        h = 1e-6 * theta[p]
        tp, tm = list(theta), list(theta)
        tp[p] += h
        tm[p] -= h
        _, Cp = ceff((tp[0], tp[1]), (tp[2], tp[3]), sc)
        _, Cm = ceff((tm[0], tm[1]), (tm[2], tm[3]), sc)
        fd = (np.sum((Cp - Ct) ** 2) - np.sum((Cm - Ct) ** 2)) / (2 * h)
        assert abs(fd - dl[p]) < 1e-5 * max(abs(dl[p]), 1e-3 * np.abs(dl).max())


def test_autograd_effective_stiffness(xf):
    """torch.autograd path: backward of ||C_eff - C_t||^2 equals the library gradient and the
    central finite difference in one Lame constant."""
    torch = pytest.importorskip("torch")
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    sc = torch.tensor(synth.voxel_scale(n, 7).ravel(), dtype=torch.float32, requires_grad=True)
    lame = torch.tensor(list(synth.lame_from_E_nu(8.0, 0.2)) + list(synth.lame_from_E_nu(1.0, 0.3)),
                        dtype=torch.float64, requires_grad=True)
    Ct = torch.tensor(np.random.default_rng(4).normal(size=(6, 6)))
    s = xf.Solver(n, tol=1e-13)
    C = xf.effective_stiffness(s, L, lame, sc)
    loss = ((C - Ct) ** 2).sum()
    loss.backward()
    dl, ds, _ = s.grad(2.0 * (C.detach().numpy() - Ct.numpy()))
    assert np.allclose(lame.grad.numpy(), dl, rtol=1e-12, atol=0)
    assert np.allclose(sc.grad.numpy(), ds, rtol=1e-6, atol=0)
    p, h = 1, 1e-6 * float(lame.detach()[1])
    with torch.no_grad():
        lp, lmn = lame.detach().clone(), lame.detach().clone()
        lp[p] += h
        lmn[p] -= h
        fp = ((xf.effective_stiffness(s, L, lp, sc.detach()) - Ct) ** 2).sum().item()
        fm = ((xf.effective_stiffness(s, L, lmn, sc.detach()) - Ct) ** 2).sum().item()
    fd = (fp - fm) / (2 * h)
    assert abs(fd - lame.grad[p].item()) < 1e-5 * abs(lame.grad[p].item())


def test_batch_uneven_microstructures(xf):
    """Batch of microstructures on uneven grids solved at once (lockstep; every inner solve of
    all contexts one device-driven graph launch), FP32-refined to 1e-8: each C_eff against its
    own FP64 solve, against the same solver run alone, and (16^3 member) against the oracle."""
    ws = synth.batch_uneven(count=6, seed=5, sizes=(16, 32, 48))
    ws[0] = dict(ws[0], n=(16, 16, 16), L=synth.sphere_levelset((16, 16, 16), (0.5, 0.5, 0.5), 0.3))
    solvers = []
    for w in ws:
        sv = xf.Solver(w["n"], precision="fp32", tol=1e-8)
        sv.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"])
        solvers.append(sv)
    Cs, sts = xf.batch_effective_stiffness(solvers)
    for w, C, st, sv in zip(ws, Cs, sts, solvers):
        s64 = xf.Solver(w["n"], precision="fp64", tol=1e-11)
        s64.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"])
        C64, st64 = s64.effective_stiffness()
        assert st64["converged"]
        assert np.abs(C - C64).max() < 1e-6 * np.abs(C64).max(), (w["n"], np.abs(C - C64).max())
        C1, st1 = sv.effective_stiffness()  # the same context alone
        assert st1["converged"]
        assert np.abs(C1 - C).max() < 1e-7 * np.abs(C).max()
    o = XFEM(ws[0]["L"], ws[0]["n"], lame_minus=ws[0]["lame_minus"], lame_plus=ws[0]["lame_plus"])
    Co, _, _ = o.effective_stiffness()
    assert np.abs(Cs[0] - Co).max() < 1e-6 * np.abs(Co).max()


def test_batch_mixed_precisions_and_schemes(xf):
    """One lockstep batch holding an FP64 context, an FP32-refined context and a nonlinear-CG
    context (their inner solves share one device-driven graph): each C_eff and iteration count
    equals that of the same context solved alone."""
    n = (16, 16, 16)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    lm, lp = synth.lame_from_E_nu(10.0, 0.3), synth.lame_from_E_nu(1.0, 0.3)
    kws = [dict(precision="fp64", tol=1e-10), dict(precision="fp32", tol=1e-8),
           dict(precision="fp64", tol=1e-9, scheme="nlcg")]
    solvers = []
    for kw in kws:
        sv = xf.Solver(n, **kw)
        sv.set_microstructure(L, lm, lp)
        solvers.append(sv)
    Cs, sts = xf.batch_effective_stiffness(solvers)
    for sv, C, st in zip(solvers, Cs, sts):
        C1, st1 = sv.effective_stiffness()
        assert st1["converged"] and st["iters"] == st1["iters"], (st["iters"], st1["iters"])
        assert np.abs(C1 - C).max() < 1e-9 * np.abs(C).max()
        sv.close()


def test_legacy_stream_matches_own_stream(xf):
    """The same solve on the legacy stream (plain launches) and on the solver's own stream
    (graph-replayed iterations) gives the same result."""
    n, ell, L, lm, lp, sc = _case("ragged")
    out = []
    for stream in ("legacy", None):
        s = xf.Solver(n, ell, precision="fp32", tol=1e-10, stream=stream)
        s.set_microstructure(L, lm, lp, sc)
        C, st = s.effective_stiffness()
        assert st["converged"]
        out.append((C, st["iters"]))
    # FP32 atomics make the sums order-dependent: equal up to rounding, not bit for bit
    assert all(abs(a - b) <= 2 for a, b in zip(out[0][1], out[1][1]))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-8 * np.abs(out[0][0]).max()


def test_laminate_closed_form_gpu(xf):
    from tests.test_oracle_pins import _laminate_closed_form
    n = (32, 32, 32)
    normal = (1, 2, 3)
    L = synth.laminate_levelset(n, normal=normal, offset=0.1234567, fraction=0.5)
    lm = synth.lame_from_E_nu(100.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    Cref = _laminate_closed_form(normal, 0.5, lm, lp)
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-6)):
        s = xf.Solver(n, precision=prec, tol=1e-11)
        s.set_microstructure(L, lm, lp)
        C, st = s.effective_stiffness()
        assert st["converged"], st
        assert np.abs(C - Cref).max() < tol * np.abs(Cref).max(), (prec, np.abs(C - Cref).max())


def _slab_modes(rng, n=(16, 128, 128)):
    """Fourier modes for an n0 x N x N grid that reach every line type of the FP32 y-z plane
    path: z frequencies 0 and N/2 (real z lines) with y frequencies 0, N/2 and others, x
    frequencies 0 and n0/2 (Nyquist), odd and even y frequencies, and generic modes."""
    h0, h = n[0] // 2, n[1] // 2
    ks = [(0, 0, 1), (1, 0, 0), (h0, 0, 0), (3, 0, h), (0, h, 0), (h0, h, h), (5, h, 0),
          (2, 7, 0), (6, h + 36, 0), (4, 9, h), (7, n[1] - 8, h), (3, h, 5), (1, 2, 3), (9, 33, 17),
          (n[0] - 1, n[1] - 1, n[2] - 1), (h0, 1, h - 1), (0, h + 13, h - 24), (11, h, h), (12, 0, h), (0, 0, h)]
    ks += [tuple(int(v) for v in rng.integers(0, n)) for _ in range(12)]
    return [(k, rng.normal(size=3) + 1j * rng.normal(size=3)) for k in ks]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_precondition_plane_waves_yz128(xf, prec):
    """y-z planes of 128 x 128 (the FP32 slab path) against the oracle's exact single-mode
    preconditioner, element by element over the whole grid."""
    n = (16, 128, 128)
    s = xf.Solver(n)
    s.set_microstructure(np.ones(n), synth.lame_from_E_nu(2.0, 0.3), synth.lame_from_E_nu(1.0, 0.3))
    o = XFEM(np.ones(n), n)
    f, zref = o.precondition_modes(_slab_modes(np.random.default_rng(11)))
    z, rr = s.precondition(f[None, :], precision=prec)
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert _rel(z[0], zref) < tol
    assert np.abs(z[0] - zref).max() < 10 * tol * np.abs(zref).max()
    assert abs(rr[0] - f @ zref) <= 10 * tol * abs(f @ zref)


@pytest.mark.parametrize("n", [(16, 32, 32), (32, 48, 48), (48, 64, 64), (16, 80, 80), (32, 96, 96),
                               (96, 48, 48)])
def test_precondition_plane_waves_square_planes(xf, n):
    """The FP32 y-z plane path at every other square plane size it serves (32 ... 96 nodes, several
    x lengths) against the oracle's exact single-mode preconditioner, element by element, with
    three right-hand sides (one x-pass group of two and a partial one)."""
    s = xf.Solver(n)
    s.set_microstructure(np.ones(n), synth.lame_from_E_nu(2.0, 0.3), synth.lame_from_E_nu(1.0, 0.3))
    o = XFEM(np.ones(n), n)
    rng = np.random.default_rng(n[1] + n[0])
    fs, zs = zip(*(o.precondition_modes(_slab_modes(rng, n)) for _ in range(3)))
    z, rr = s.precondition(np.stack(fs), precision="fp32")
    for k in range(3):
        assert _rel(z[k], zs[k]) < 2e-5, (n, k)
        assert np.abs(z[k] - zs[k]).max() < 2e-4 * np.abs(zs[k]).max()
        assert abs(rr[k] - fs[k] @ zs[k]) <= 2e-4 * abs(fs[k] @ zs[k])


def test_laminate_closed_form_yz128(xf):
    """Full FP32-refined solve through the y-z plane path: planar interface, exact C_eff."""
    from tests.test_oracle_pins import _laminate_closed_form
    n = (16, 128, 128)
    normal = (1, 2, 3)
    L = synth.laminate_levelset(n, normal=normal, offset=0.1234567, fraction=0.5)
    lm = synth.lame_from_E_nu(100.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    Cref = _laminate_closed_form(normal, 0.5, lm, lp)
    s = xf.Solver(n, precision="fp32", tol=1e-11)
    s.set_microstructure(L, lm, lp)
    C, st = s.effective_stiffness()
    assert st["converged"], st
    assert np.abs(C - Cref).max() < 1e-6 * np.abs(Cref).max(), np.abs(C - Cref).max()


def test_full_size_laminate_384(xf):
    """Precision at scale: the 384^3 laminate tilted by (1,2,3)/sqrt(14), contrast 100,
    FP32-refined, against its closed-form C_eff to 1e-6 (the X-FEM solution is exact for a
    laminate, so the closed form holds at any grid size)."""
    from tests.test_oracle_pins import _laminate_closed_form
    w = synth.make_workload("laminate")
    s = xf.Solver(w["n"], precision="fp32", tol=1e-9)
    s.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"])
    C, st = s.effective_stiffness()
    assert st["converged"], st
    Cref = _laminate_closed_form(w["info"]["normal"], w["info"]["fraction"], w["lame_minus"], w["lame_plus"])
    assert np.abs(C - Cref).max() < 1e-6 * np.abs(Cref).max(), np.abs(C - Cref).max()


def test_full_size_fibers_256(xf):
    """Precision at scale: 256^3 with 60 periodic fibers (contrast 100): FP32-refined against plain
    FP64 to 1e-6; C_eff symmetric, positive definite and between the Reuss and Voigt bounds of the
    phase volume fractions (properties that hold at any size)."""
    from oracle import iso_stiffness
    w = synth.make_workload("fibers60")
    out = {}
    for prec, tol in (("fp32", 1e-8), ("fp64", 1e-10)):
        s = xf.Solver(w["n"], precision=prec, tol=tol)
        s.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"])
        out[prec], st = s.effective_stiffness()
        assert st["converged"], (prec, st)
        s.close()
    C, C64 = out["fp32"], out["fp64"]
    assert np.abs(C - C64).max() < 1e-6 * np.abs(C64).max(), np.abs(C - C64).max()
    assert np.abs(C64 - C64.T).max() < 1e-8 * np.abs(C64).max()
    assert np.linalg.eigvalsh(0.5 * (C64 + C64.T)).min() > 0.0
    f = float(np.mean(w["L"] < 0.0))  # nodal estimate of the fibre fraction
    Ci, Cm = iso_stiffness(*w["lame_minus"]), iso_stiffness(*w["lame_plus"])
    voigt = f * Ci + (1 - f) * Cm
    reuss = np.linalg.inv(f * np.linalg.inv(Ci) + (1 - f) * np.linalg.inv(Cm))
    sym = 0.5 * (C64 + C64.T)
    assert np.linalg.eigvalsh(voigt - sym).min() > -1e-2 * np.abs(C64).max()
    assert np.linalg.eigvalsh(sym - reuss).min() > -1e-2 * np.abs(C64).max()


def test_full_size_apply_and_precondition_128(xf):
    """The bench workload at its full size (128^3, 40 ellipsoids, voxel scale), in the kernels'
    bench launch shapes: the preconditioner on a superposition of Fourier modes against the
    oracle's exact values everywhere (enriched part: identity), and the stiffness operator's
    properties - symmetry, rigid translations in its kernel, FP32 and double-word applies
    against FP64."""
    w = synth.make_workload("ellipsoids40")
    n = w["n"]
    s = xf.Solver(n)
    s.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"], w["scale"])
    N, nX = int(np.prod(n)), s.num_enriched
    rng = np.random.default_rng(21)
    og = XFEM(np.ones(n), n)
    ks = [(0, 0, 1), (64, 0, 0), (3, 64, 0), (0, 5, 64), (64, 64, 64), (7, 100, 3), (127, 1, 33), (20, 0, 64)]
    ks += [tuple(int(v) for v in rng.integers(0, 128, 3)) for _ in range(6)]
    f_std, z_std = og.precondition_modes([(k, rng.normal(size=3) + 1j * rng.normal(size=3)) for k in ks])
    f = np.concatenate([f_std, rng.normal(size=3 * nX)])[None, :]
    for prec, tol in (("fp64", 1e-11), ("fp32", 2e-5)):
        z, rr = s.precondition(f, precision=prec)
        assert _rel(z[0, : 3 * N], z_std) < tol, prec
        assert _rel(z[0, 3 * N:], f[0, 3 * N:]) < tol, prec
    x = rng.normal(size=(2, 3 * (N + nX)))
    Ax, _ = s.apply(x, precision="fp64")
    assert abs(x[0] @ Ax[1] - x[1] @ Ax[0]) < 1e-11 * abs(x[0] @ Ax[1]) + 1e-12 * np.linalg.norm(Ax[0]) * np.linalg.norm(x[1])
    t = np.zeros((1, 3 * (N + nX)))
    t[0, N: 2 * N] = 1.0  # rigid translation along y
    At, _ = s.apply(t, precision="fp64")
    assert np.linalg.norm(At) < 1e-11 * np.linalg.norm(Ax[0]) * np.linalg.norm(t) / np.linalg.norm(x[0])
    for prec, tol in (("dw", 1e-11), ("fp32", 2e-5)):
        Ap, _ = s.apply(x, precision=prec)
        assert _rel(Ap, Ax) < tol, prec


def test_full_size_spheres27_64(xf):
    """Config 2 at full size (64^3, 27 spheres, vf 20 %, contrast 100, six load cases): C_eff
    against the oracle's (tests/golden/spheres27_64_ceff.json, written from oracle/ alone by
    make_spheres27_ceff.py), FP64 to 1e-9 and FP32-refined to 1e-6; the setup counts exactly."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "spheres27_64_ceff.json")))
    Cg = np.array(gold["C_stress"])
    w = synth.make_workload("spheres27")
    for prec, tol, bar in (("fp64", 1e-12, 1e-9), ("fp32", 1e-9, 1e-6)):
        s = xf.Solver(w["n"], precision=prec, tol=tol)
        s.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"])
        assert s.num_enriched == gold["n_enriched"] and s.num_cut_tets == gold["n_cut_tets"]
        C, st = s.effective_stiffness()
        assert st["converged"], (prec, st)
        assert np.abs(C - Cg).max() < bar * np.abs(Cg).max(), (prec, np.abs(C - Cg).max())
        s.close()


def test_full_size_gradient_128(xf):
    """Differentiation at full size: 128^3, 40 ellipsoids, per-voxel modulus scale, loss
    ||C_eff - C_t||^2.  The FP64 adjoint against central finite differences (h = 1e-6 relative,
    FP64 solves) in one Lame constant of each phase; the FP32-refined gradient against the FP64
    one."""
    w = synth.make_workload("ellipsoids40")
    n, L, sc = w["n"], w["L"], w["scale"]
    theta = [*w["lame_minus"], *w["lame_plus"]]

    def solve(th, prec="fp64", tol=1e-12):
        s = xf.Solver(n, precision=prec, tol=tol)
        s.set_microstructure(L, (th[0], th[1]), (th[2], th[3]), sc)
        C, st = s.effective_stiffness()
        assert st["converged"], st
        return s, C

    s64, C0 = solve(theta)
    G = np.random.default_rng(4).normal(size=(6, 6))
    G = 0.5 * (G + G.T)
    Ct = C0 + 0.05 * np.linalg.norm(C0) / np.linalg.norm(G) * G
    dl, ds, _ = s64.grad(2.0 * (C0 - Ct))
    s64.close()
    for p in (0, 3):
        h = 1e-6 * theta[p]
        tp, tm = list(theta), list(theta)
        tp[p] += h
        tm[p] -= h
        sp_, Cp = solve(tp)
        sp_.close()
        sm_, Cm = solve(tm)
        sm_.close()
        fd = (np.sum((Cp - Ct) ** 2) - np.sum((Cm - Ct) ** 2)) / (2 * h)
        assert abs(fd - dl[p]) < 1e-5 * np.abs(dl).max(), (p, fd, dl[p])
    s32, C32 = solve(theta, "fp32", 1e-8)
    dl32, ds32, _ = s32.grad(2.0 * (C32 - Ct))
    assert np.abs(dl32 - dl).max() < 1e-5 * np.abs(dl).max()
    assert _rel(ds32.astype(np.float64), ds.astype(np.float64)) < 1e-4


def test_dw_residual_suffices_at_high_contrast_128(xf):
    """The refinement's residual uses the plain double-word sum (no relative bound under
    cancellation).  At 128^3 (the bench's ellipsoids) with contrast 1000 and tol 1e-10 the
    FP32-refined solve still converges and its mean stress equals a plain FP64 solve's to 1e-9:
    the residual's rounding stays below the tolerance there."""
    w = synth.make_workload("ellipsoids40")
    lm, lp = synth.lame_from_E_nu(1000.0, 0.2), synth.lame_from_E_nu(1.0, 0.3)
    e = np.eye(6)[:1]
    out = {}
    for prec in ("fp32", "fp64"):
        s = xf.Solver((128, 128, 128), precision=prec, tol=1e-10, maxit=20000)
        s.set_microstructure(w["L"], lm, lp, w["scale"])
        out[prec] = s.solve(e, u=False)
        s.close()
    assert out["fp32"]["converged"] and out["fp64"]["converged"]
    assert out["fp32"]["stats"]["final_res"][0] <= 1e-10
    a, b = out["fp32"]["mean_stress"][0], out["fp64"]["mean_stress"][0]
    assert np.abs(a - b).max() < 1e-9 * np.abs(b).max(), np.abs(a - b).max() / np.abs(b).max()


def test_homogeneous_and_equal_phase_edge_cases(xf):
    n = (4, 4, 4)
    lp = synth.lame_from_E_nu(2.0, 0.3)
    s = xf.Solver(n)
    s.set_microstructure(np.ones(n), (5.0, 1.0), lp)
    assert s.num_enriched == 0 and s.num_cut_tets == 0
    C, st = s.effective_stiffness()
    from oracle import iso_stiffness
    assert np.allclose(C, iso_stiffness(*lp), atol=1e-13)
    n = (8, 8, 8)
    lam = synth.lame_from_E_nu(3.0, 0.25)
    L = synth.sphere_levelset(n, (0.43, 0.51, 0.47), 0.27)
    s = xf.Solver(n)
    s.set_microstructure(L, lam, lam)
    assert s.num_enriched > 0
    out = s.solve(np.eye(6))
    assert np.abs(out["u_std"]).max() < 1e-11
    assert np.allclose(out["mean_stress"], iso_stiffness(*lam), atol=1e-12)


def test_invalid_arguments_are_reported(xf):
    with pytest.raises(xf.XfftError):
        xf.Solver((7, 8, 8))
    with pytest.raises(xf.XfftError):
        xf.Solver((14, 8, 8))  # 7 is not a supported radix
    s = xf.Solver((8, 8, 8))
    with pytest.raises(xf.XfftError):
        s.solve(np.eye(6)[:1])  # before set_microstructure
    with pytest.raises(xf.XfftError):
        s.set_microstructure(np.ones((8, 8, 8)), (1.0, -1.0), (1.0, 1.0))


@pytest.mark.parametrize("tol", [1e-8, 1e-11])
def test_residual_update_equals_recomputed_residuals(xf, tol):
    """Iterative refinement with the residual update (default: once the residual is below 100 tol,
    r_k = r_{k-1} - A delta_k with the FP32 operator on the correction) against every residual
    recomputed in double-word arithmetic: the same C_eff to well inside the tolerance, both
    converged, and both against a plain FP64 solve.  On the 64^3 ellipsoids (per-voxel scale),
    where the refinement takes at least two steps."""
    w = synth.make_workload("ellipsoids40", n=(64, 64, 64))
    out = {}
    for upd in (True, False):
        s = xf.Solver((64, 64, 64), precision="fp32", tol=tol, residual_update=upd)
        s.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"], w["scale"])
        C, st = s.effective_stiffness()
        assert st["converged"], (upd, st)
        out[upd] = (C, st)
        s.close()
    s64 = xf.Solver((64, 64, 64), precision="fp64", tol=min(tol, 1e-10))
    s64.set_microstructure(w["L"], w["lame_minus"], w["lame_plus"], w["scale"])
    C64, st64 = s64.effective_stiffness()
    assert st64["converged"]
    (Cu, stu), (Cr, str_) = out[True], out[False]
    sc = np.abs(C64).max()
    assert stu["refine_steps"] >= 1 and str_["refine_steps"] >= 1, (stu, str_)
    assert np.abs(Cu - Cr).max() < 10 * tol * sc, np.abs(Cu - Cr).max() / sc
    assert np.abs(Cu - C64).max() < 10 * tol * sc + 1e-10 * sc, np.abs(Cu - C64).max() / sc


def _axis_modes(rng, n):
    """Fourier modes of an n0 x n1 x n2 grid: zero and Nyquist frequencies on each axis and in
    combination, odd frequencies, and random ones."""
    h = [m // 2 for m in n]
    ks = [(0, 0, 1), (1, 0, 0), (0, 1, 0), (h[0], 0, 0), (0, h[1], 0), (0, 0, h[2]), (h[0], h[1], h[2]),
          (3, 5, 7), (h[0] - 1, 1, h[2]), (1, h[1] + 3, 2), (n[0] - 1, n[1] - 1, n[2] - 1), (5, 0, h[2] + 1)]
    ks += [tuple(int(v) for v in rng.integers(0, n)) for _ in range(12)]
    return [(k, rng.normal(size=3) + 1j * rng.normal(size=3)) for k in ks]


@pytest.mark.parametrize("n", [(384, 16, 16), (16, 384, 16), (16, 16, 384)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_precondition_plane_waves_384(xf, n, prec):
    """Lines of 384 points (the plan 4 x 4 x 4 x 6 with the radix-6 butterfly) along each axis:
    the preconditioner against the oracle's exact single-mode values, element by element (x:
    the y-z plane path's x pass; y, z: the five-pass kernels)."""
    s = xf.Solver(n)
    s.set_microstructure(np.ones(n), synth.lame_from_E_nu(2.0, 0.3), synth.lame_from_E_nu(1.0, 0.3))
    o = XFEM(np.ones(n), n)
    f, zref = o.precondition_modes(_axis_modes(np.random.default_rng(sum(n)), n))
    z, rr = s.precondition(f[None, :], precision=prec)
    tol = 1e-11 if prec == "fp64" else 2e-5
    assert _rel(z[0], zref) < tol
    assert np.abs(z[0] - zref).max() < 10 * tol * np.abs(zref).max()
    assert abs(rr[0] - f @ zref) <= 10 * tol * abs(f @ zref)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "dw"])
def test_apply_matches_oracle_several_tiles(xf, prec):
    """Element-wise parity of the apply on a 96 x 48 x 32 grid: three 32-plane x chunks of the
    stencil's x-marching, four y tiles and three z tiles of 15 owned nodes with ragged last
    tiles, two inclusions and a per-voxel scale, against the oracle's assembled operator."""
    n, ell, L, lm, lp, sc = _case("tiles")
    s = xf.Solver(n, ell)
    s.set_microstructure(L, lm, lp, sc)
    o = _oracle("tiles")
    o.assemble()
    rng = np.random.default_rng(12)
    d = rng.normal(size=(2, o.ndof))
    eps = rng.normal(size=(2, 6))
    tol = {"fp64": 1e-12, "dw": 1e-11, "fp32": 2e-5}[prec]
    q, _ = s.apply(d, precision=prec)
    for r in range(2):
        ref = o.A @ d[r]
        assert _rel(q[r], ref) < tol
        assert np.abs(q[r] - ref).max() < 20 * tol * np.abs(ref).max()
    q, sig = s.apply(d, eps=eps, precision=prec)
    for r in range(2):
        assert _rel(q[r], o.A @ d[r] + o.rhs(eps[r])) < tol
        assert _rel(sig[r], np.asarray(o.Sm @ d[r]).ravel() + o.Cbar @ eps[r]) < tol
