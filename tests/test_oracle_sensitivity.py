"""The oracle's closed-form pins catch plausible mistakes (no GPU needed).

Each test plants one mistake in the oracle, on the CPU and only inside the test, and checks that
the laminate closed form it would otherwise meet to rounding (exact because the laminate's
solution lies in the X-FEM space) now fails by far more than the pin's tolerance.  A change of
basis that the method allows (the enrichment scaling D0 per node instead of per DOF; eq.
XFFT_diagonal leaves this open) is the negative control: the pin still holds.
"""
import numpy as np

import synth
from oracle import XFEM, symgrad_operator
from test_oracle_pins import _laminate_closed_form

LM = synth.lame_from_E_nu(10.0, 0.2)
LP = synth.lame_from_E_nu(1.0, 0.3)
PH3 = [synth.lame_from_E_nu(10.0, 0.2), synth.lame_from_E_nu(1.0, 0.3), synth.lame_from_E_nu(3.0, 0.4)]


def _ceff(o):
    o.assemble()
    C = np.zeros((6, 6))
    for k in range(6):
        e = np.eye(6)[k]
        C[:, k] = o.mean_stress(o.solve_direct(e), e)
    return C


def _laminate_error(**kw):
    """Tilted two-phase laminate (normal (1,0,1), 8^3): relative max error of C_eff."""
    normal = (1, 0, 1)
    n = (8, 8, 8)
    L = synth.laminate_levelset(n, normal=normal, offset=0.137, fraction=0.5)
    C = _ceff(XFEM(L, n, lame_minus=LM, lame_plus=LP, **kw))
    Cref = _laminate_closed_form(normal, 0.5, LM, LP)
    return np.abs(C - Cref).max() / np.abs(Cref).max()


def _three_layer_error():
    """Three layers (normal (1,0,0), 8^3, two level sets): relative max error of C_eff."""
    fr = (0.36, 0.32, 0.32)
    n = (8, 8, 8)
    L0 = synth.laminate_levelset(n, normal=(1, 0, 0), offset=0.137, fraction=fr[0])
    L1 = synth.laminate_levelset(n, normal=(1, 0, 0), offset=0.137 + fr[0] / 2, fraction=fr[0] / 2 + fr[1])
    C = _ceff(XFEM(np.stack([L0, L1]), n, phases=PH3))
    Cref = _laminate_closed_form((1, 0, 0), None, None, None, layers=list(zip(fr, PH3)))
    return np.abs(C - Cref).max() / np.abs(Cref).max()


def test_unplanted_pins_hold():
    assert _laminate_error() < 1e-12
    assert _three_layer_error() < 1e-12


def test_wrong_side_sign_of_the_enrichment(monkeypatch):
    """rho restricted to side s built with |L| + s L instead of |L| - s L."""
    orig = XFEM._enriched_B
    monkeypatch.setattr(XFEM, "_enriched_B", lambda self, G, Lv, s, bary: orig(self, G, Lv, -s, bary))
    assert _laminate_error() > 1e-3


def test_dropped_product_rule_term(monkeypatch):
    """grad(N_a rho) = rho grad N_a + N_a grad rho with the second term dropped."""
    def bad(self, G, Lv, s, bary):
        rho = bary @ (np.abs(Lv) - s * Lv)
        return symgrad_operator(rho[:, None, None] * G[None, :, :])
    monkeypatch.setattr(XFEM, "_enriched_B", bad)
    assert _laminate_error() > 1e-3


def test_cut_tet_sides_with_swapped_phases(monkeypatch):
    monkeypatch.setattr(XFEM, "_side_phase", lambda self, idx, s: int(self.cut_phase[-s][idx]))
    assert _laminate_error() > 1e-3


def test_plus_side_always_the_last_phase(monkeypatch):
    """Several interfaces: the plus side of every cut tet taken as phase K (the matrix)."""
    orig = XFEM._classify

    def bad(self):
        orig(self)
        self.cut_phase = {-1: self.cut_phase[-1], +1: np.full_like(self.cut_phase[+1], self.nL)}
    monkeypatch.setattr(XFEM, "_classify", bad)
    assert _three_layer_error() > 1e-3


def test_snap_threshold_in_the_wrong_units():
    """tau = 0.3 h instead of 1e-6 h moves the interface where nodes lie close to it."""
    assert _laminate_error(tau=0.3 / 8) > 1e-4


def test_enrichment_scaling_per_node_is_a_change_of_basis(monkeypatch):
    """Negative control: D0 per node (the trace of the per-DOF 3 x 3 block, the same value for
    the three components) instead of per DOF changes the basis only, so C_eff is unchanged."""
    orig = XFEM._cut_quadrature

    def per_node(self):
        orig(self)
        if self.nX:
            self.D = np.repeat(self.D.sum(axis=1, keepdims=True), 3, axis=1)
            self.Dinvsqrt = 1.0 / np.sqrt(self.D)
    monkeypatch.setattr(XFEM, "_cut_quadrature", per_node)
    assert _laminate_error() < 1e-12
