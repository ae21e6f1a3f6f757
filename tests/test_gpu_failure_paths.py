"""Failure paths of the C-ABI, driven by host-made inputs only (nothing here faults, traps or
hangs the GPU): non-finite inputs are refused, an iteration cap returns XFFT_ENOTCONV with the
last iterate in the outputs, an indefinite operator is caught by the device-side check of
<A d, d> (XFFT_EBREAKDOWN), and an allocation cap returns XFFT_ENOMEM and leaks nothing."""
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


def _case():
    n = (12, 12, 12)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    return n, L, synth.lame_from_E_nu(10.0, 0.3), synth.lame_from_E_nu(1.0, 0.3)


def test_non_finite_inputs_are_refused(xf):
    n, L, lm, lp = _case()
    s = xf.Solver(n)
    for bad in (np.nan, np.inf, -np.inf):
        Lb = L.copy()
        Lb[3, 4, 5] = bad
        with pytest.raises(xf.XfftError) as ei:
            s.set_microstructure(Lb, lm, lp)
        assert ei.value.status == xf.capi.XFFT_EINVAL and "level set" in str(ei.value)
    sc = np.ones(n, dtype=np.float32)
    sc[0, 0, 7] = np.nan
    with pytest.raises(xf.XfftError) as ei:
        s.set_microstructure(L, lm, lp, sc)
    assert ei.value.status == xf.capi.XFFT_EINVAL and "scale" in str(ei.value)
    # an indefinite phase (lambda < -2 mu / 3) is refused on the host
    with pytest.raises(xf.XfftError) as ei:
        s.set_microstructure(L, (-1.0, 1.0), lp)
    assert ei.value.status == xf.capi.XFFT_EINVAL
    # the context stays usable
    s.set_microstructure(L, lm, lp)
    assert s.solve(np.eye(6)[:1], u=False)["converged"]
    s.close()


def test_iteration_cap_returns_the_last_iterate(xf):
    """maxit = 1: XFFT_ENOTCONV, and the outputs hold the iterate after one CG step, which is
    the oracle's one-step PCG iterate (both standard and unscaled enriched parts)."""
    n, L, lm, lp = _case()
    e = np.array([0.3, -0.1, 0.2, 0.05, 0.1, -0.2])
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp)
    u1, info = o.pcg(e, tol=1e-12, maxit=1, green="fft")
    assert info["iters"] == 1 and not info["converged"]
    for prec in ("fp64", "fp32"):
        s = xf.Solver(n, precision=prec, tol=1e-12, maxit=1, max_refine=1)
        s.set_microstructure(L, lm, lp)
        _, st = s.effective_stiffness()  # XFFT_ENOTCONV is returned as converged = False
        assert not st["converged"]
        out = s.solve(e[None], u=True)
        assert not out["converged"]
        if prec == "fp64":
            assert out["stats"]["iters"][0] == 1
            us = u1[: 3 * o.nFE].reshape(3, -1)
            ue = u1[3 * o.nFE:].reshape(3, -1) * o.Dinvsqrt.T
            assert np.linalg.norm(out["u_std"][0] - us) < 1e-10 * np.linalg.norm(us)
            assert np.linalg.norm(out["u_enr"][0] - ue) < 1e-10 * np.linalg.norm(ue)
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_indefinite_operator_is_caught_on_the_device(xf, prec):
    """A negative modulus scale (finite, so accepted by set_microstructure) makes A negative
    definite: the first <A d, d> is negative and the device-side check stops the right-hand
    side with XFFT_EBREAKDOWN; the context stays usable."""
    n, L, lm, lp = _case()
    s = xf.Solver(n, precision=prec)
    s.set_microstructure(L, lm, lp, -np.ones(n, dtype=np.float32))
    with pytest.raises(xf.XfftError) as ei:
        s.solve(np.eye(6)[:2], u=False)
    assert ei.value.status == xf.capi.XFFT_EBREAKDOWN
    s.set_microstructure(L, lm, lp)
    assert s.solve(np.eye(6)[:1], u=False)["converged"]
    s.close()


def test_allocation_cap_returns_enomem_and_leaks_nothing(xf):
    import torch
    n, L, lm, lp = _case()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for cap in (4096, 1_000_000):  # set_microstructure fails, or the solver workspace does
        s = xf.Solver(n, max_device_bytes=cap)
        with pytest.raises(xf.XfftError) as ei:
            s.set_microstructure(L, lm, lp)
            s.effective_stiffness()
        assert ei.value.status == xf.capi.XFFT_ENOMEM
        s.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= 4 << 20, (free0, free1)
    # the same solver without the cap works
    s = xf.Solver(n)
    s.set_microstructure(L, lm, lp)
    assert s.effective_stiffness()[1]["converged"]
    s.close()


def test_device_loop_time_limit_returns_etimeout(xf):
    """spin_limit_ns = 0: the device-driven iteration loop stops after its first round and the
    call returns XFFT_ETIMEOUT with the last iterate; nothing is left running on the GPU (the
    stream drains) and the same microstructure then converges without the limit, in a single
    solve and in a lockstep batch."""
    import torch
    n, L, lm, lp = _case()
    for prec in ("fp64", "fp32"):
        s = xf.Solver(n, precision=prec, tol=1e-10, spin_limit_ns=0)
        s.set_microstructure(L, lm, lp)
        with pytest.raises(xf.XfftError) as ei:
            s.solve(np.eye(6)[:2], u=False)
        assert ei.value.status == xf.capi.XFFT_ETIMEOUT
        torch.cuda.synchronize()
        s2 = xf.Solver(n, precision=prec, tol=1e-10)
        s2.set_microstructure(L, lm, lp)
        assert s2.solve(np.eye(6)[:2], u=False)["converged"]
        with pytest.raises(xf.XfftError) as ei:
            xf.batch_effective_stiffness([s, s2])
        assert ei.value.status == xf.capi.XFFT_ETIMEOUT
        torch.cuda.synchronize()
        C, st = xf.batch_effective_stiffness([s2])
        assert st[0]["iters"][0] > 0
        s.close()
        s2.close()
