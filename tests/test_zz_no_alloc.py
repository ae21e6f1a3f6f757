"""The allocation-free apply (xfft_apply_noalloc) against the allocating xfft_apply.

For callers that must not allocate device memory while running (their memory belongs to their
own pool allocator, or a cudaMalloc's implicit device synchronisation is not acceptable).  Its
reduction scratch is a fixed device array shared by all calls, so two calls in a row must both
give the same results as the allocating entry point.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_apply_noalloc_matches_apply_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_02172_gb300 import Solver

    n = (10, 12, 8)
    L = np.minimum(synth.sphere_levelset(n, (0.3, 0.4, 0.5), 0.22),
                   synth.sphere_levelset(n, (0.8, 0.85, 0.2), 0.15))
    s = Solver(n)
    s.set_microstructure(L, synth.lame_from_E_nu(20.0, 0.2), synth.lame_from_E_nu(1.0, 0.3),
                         synth.voxel_scale(n, 3))
    rng = np.random.default_rng(17)
    k = 3
    d_h = rng.normal(size=(k, s.stride))
    q_ref, sig_ref = s.apply(d_h)  # the allocating entry point
    d = torch.from_numpy(d_h).cuda()
    for call in range(2):
        q = torch.full_like(d, float("nan"))
        out = torch.full((k, 7), float("nan"), dtype=torch.float64, device="cuda")
        s.apply_noalloc(d, q, out)
        torch.cuda.synchronize()
        qn = q.cpu().numpy()
        on = out.cpu().numpy()
        for r in range(k):
            assert np.linalg.norm(qn[r] - q_ref[r]) <= 1e-12 * np.linalg.norm(q_ref[r]), call
            assert np.abs(on[r, 1:] - sig_ref[r]).max() <= 1e-12 * np.abs(sig_ref[r]).max(), call
            dad = float(d_h[r] @ q_ref[r])
            assert abs(on[r, 0] - dad) <= 1e-12 * abs(dad), call
    s.close()


def test_apply_noalloc_refuses_requests_beyond_its_scratch():
    """More right-hand sides than XFFT_NOALLOC_MAX_RHS, or a grid whose apply launches more than
    XFFT_NOALLOC_MAX_PARTS blocks (384^3: 26 x 26 x 12 stencil blocks), return XFFT_EINVAL and
    leave the output untouched."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_02172_gb300 import Solver, XfftError, capi

    n = (10, 12, 8)
    s = Solver(n)
    s.set_microstructure(synth.sphere_levelset(n, (0.3, 0.4, 0.5), 0.22),
                         synth.lame_from_E_nu(20.0, 0.2), synth.lame_from_E_nu(1.0, 0.3))
    k = capi.NOALLOC_MAX_RHS + 1
    d = torch.ones((k, s.stride), dtype=torch.float64, device="cuda")
    q = torch.full_like(d, float("nan"))
    with pytest.raises(XfftError) as ei:
        s.apply_noalloc(d, q)
    assert ei.value.status == capi.XFFT_EINVAL
    torch.cuda.synchronize()
    assert bool(torch.isnan(q).all())
    s.close()
    n = (384, 384, 384)
    s = Solver(n)
    s.set_microstructure(np.ones(n), (1.0, 1.0), (1.0, 1.0))
    d = torch.zeros((1, s.stride), dtype=torch.float64, device="cuda")
    q = torch.full_like(d, float("nan"))
    with pytest.raises(XfftError) as ei:
        s.apply_noalloc(d, q)
    assert ei.value.status == capi.XFFT_EINVAL
    torch.cuda.synchronize()
    assert bool(torch.isnan(q).all())
    s.close()
