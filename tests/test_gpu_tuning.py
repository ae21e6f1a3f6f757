"""The launch-shape tuner of the FP32 cut-tet kernel (north star: "tile shapes picked by a
project-written autotuner"): the picked grid and right-hand sides per launch are among the
candidates, the tuned solve equals the untuned one to the FP32-refined tolerance, the choice is
reused for the same microstructure, and the partial sums stay consistent (the same C_eff as the
oracle on a small grid)."""
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


def test_tuned_launch_shape_matches_defaults(xf):
    w = synth.make_workload("ellipsoids40", n=(64, 64, 64))
    lm, lp = w["lame_minus"], w["lame_plus"]
    Cs, shapes = [], []
    for tune in (False, True, True):
        s = xf.Solver((64, 64, 64), precision="fp32", tol=1e-8, autotune=tune)
        s.set_microstructure(w["L"], lm, lp, w["scale"])
        C, st = s.effective_stiffness()
        assert st["converged"]
        Cs.append(C)
        shapes.append(s.tuning)
        ncut = s.num_cut_tets
        s.close()
    nb_max = min(-(-ncut // 128), 2432)
    blocks, rpl, group = shapes[1]
    assert rpl in (3, 6) and 152 <= blocks <= max(nb_max, 1216) and group in (1, 2, 3, 64), shapes
    assert shapes[2] == shapes[1]             # the cached choice for the same microstructure
    assert shapes[0][1:] == (8, 64)           # untuned: all right-hand sides in one launch
    assert np.abs(Cs[1] - Cs[0]).max() < 1e-6 * np.abs(Cs[0]).max()


def test_tuned_solve_matches_oracle(xf):
    n = (16, 16, 16)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.33)
    lm, lp = synth.lame_from_E_nu(20.0, 0.2), synth.lame_from_E_nu(1.0, 0.3)
    s = xf.Solver(n, precision="fp32", tol=1e-9)
    s.set_microstructure(L, lm, lp)
    e = np.array([[0.2, -0.1, 0.3, 0.4, -0.2, 0.1]])
    out = s.solve(np.repeat(e, 6, axis=0), u=False)
    assert out["converged"]
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    ms = o.mean_stress(o.solve_direct(e[0]), e[0])
    assert np.abs(out["mean_stress"] - ms).max() < 1e-6 * np.abs(ms).max()
