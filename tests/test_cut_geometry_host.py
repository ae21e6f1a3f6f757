"""The CUDA path's per-tet setup geometry, compiled for the host (no GPU), against the oracle.

`csrc/cut_geometry.cuh` holds the classification of a tet against K level sets and the exact
side moments int N_b, int N_b N_c of a cut tet (case table of the linearised interface, Sec. 3,
Fig. subdivision).  Here it is built into a host library and compared with the oracle's generic
convex clip and 4-point quadrature, on random tets including snapped zero vertices, and with
the oracle's phase rule for several interfaces; the closed-form scaled element matrix of the
optional cut-tet cache is compared with the oracle's quadrature-assembled element matrices.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import XFEM, clip_tet, quad4

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

pytestmark = pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")


@pytest.fixture(scope="module")
def geo(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("hostgeo") / "libcutgeo.so")
    src = os.path.join(ROOT, "tests", "host", "cut_geometry_host.cu")
    inc = ["-I" + os.path.join(ROOT, "paper_2601_02172_gb300", "csrc"), "-I" + os.path.join(ROOT, "include")]
    subprocess.run([NVCC, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC"]
                   + inc + ["-o", out, src], check=True, capture_output=True)
    lib = C.CDLL(out)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    lib.host_side_moments.argtypes = [dp, C.c_int, C.c_double, dp, dp]
    lib.host_classify_tet.argtypes = [dp, C.c_int, ip, ip, ip]
    lib.host_classify_tet.restype = C.c_uint
    lib.host_cut_element_matrix.argtypes = [dp, C.c_int, dp, dp, dp, dp, dp, dp]
    lib.host_cut_scaling.argtypes = [dp, C.c_int, dp, dp, dp, dp, dp]
    lib.host_block_inverse.argtypes = [dp, dp]
    lib.host_block_inverse.restype = C.c_int
    return lib


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _oracle_moments(L, s):
    """int_side N_b and int_side N_b N_c on the reference tet (volume 1/6) from the oracle's
    clip and quadrature."""
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    qb, qw = quad4()
    m = np.zeros(4)
    M = np.zeros((4, 4))
    for P in clip_tet(X, L, s):
        vol = abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6.0
        pts = qb @ P
        bary = np.column_stack([1.0 - pts.sum(axis=1), pts])
        w = qw * vol
        m += w @ bary
        M += np.einsum("q,qb,qc->bc", w, bary, bary)
    return m, M


PACK = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def test_side_moments_match_the_oracle_clip(geo):
    rng = np.random.default_rng(7)
    cases = [rng.normal(size=4) for _ in range(300)]
    # snapped zero vertices: one or two zeros with both signs among the others
    for _ in range(100):
        L = rng.normal(size=4)
        L[rng.choice(4, size=rng.integers(1, 3), replace=False)] = 0.0
        cases.append(L)
    n = 0
    for L in cases:
        if not (L.min() < 0.0 < L.max()):
            continue
        n += 1
        for s in (+1, -1):
            m = np.zeros(4)
            Mp = np.zeros(10)
            geo.host_side_moments(_ptr(np.ascontiguousarray(L)), s, 1.0 / 6.0, _ptr(m), _ptr(Mp))
            mo, Mo = _oracle_moments(L, s)
            assert np.allclose(m, mo, atol=1e-14), (L, s)
            assert np.allclose(Mp, [Mo[b, c] for b, c in PACK], atol=1e-14), (L, s)
    assert n > 250


def test_classification_matches_the_oracle_phase_rule(geo):
    """Random vertex values of K = 1 or 2 level sets (with zeros): the tet code, the side phases
    of cut tets and the two-interface refusal agree with the oracle's rule."""
    rng = np.random.default_rng(11)
    seen = set()
    for _ in range(2000):
        K = int(rng.integers(1, 3))
        Lv = np.round(rng.normal(size=(K, 4)), 1)  # many exact zeros
        pm, pp, two = C.c_int(), C.c_int(), C.c_int()
        code = geo.host_classify_tet(_ptr(np.ascontiguousarray(Lv)), K, C.byref(pm), C.byref(pp), C.byref(two))
        neg = Lv.min(axis=1) < 0.0
        pos = Lv.max(axis=1) > 0.0
        first = int(np.argmax(neg)) if neg.any() else K
        cut = first < K and pos[first]
        if cut:
            later = [l for l in range(first + 1, K) if neg[l]]
            exp_two = any(pos[l] for l in later)
            assert code == 2 and pm.value == first and bool(two.value) == exp_two
            if not exp_two:
                assert pp.value == (later[0] if later else K)
            seen.add(("cut", first, exp_two))
        else:
            assert code == (3 if first == 2 else first) and not two.value
            seen.add(("uncut", first))
    assert ("cut", 0, True) in seen and ("cut", 1, False) in seen and ("uncut", 2) in seen


def test_cut_element_matrix_matches_the_oracle(geo):
    """The cached element matrix (closed form from the side moments, FP64 before the FP32 store)
    against the oracle's element matrices on a sphere with a voxel scale field."""
    n = (8, 8, 8)
    L = synth.sphere_levelset(n, (0.45, 0.5, 0.55), 0.3)
    lm = synth.lame_from_E_nu(8.0, 0.2)
    lp = synth.lame_from_E_nu(1.0, 0.3)
    sc = synth.voxel_scale(n, 3).astype(np.float64)
    o = XFEM(L, n, lame_minus=lm, lame_plus=lp, scale=sc)
    vol = float(np.prod(o.h)) / 6.0
    iu = np.triu_indices(24)
    worst = 0.0
    for idx in range(0, len(o.cut_list), 3):
        v, t = o.cut_list[idx]
        Lv = np.ascontiguousarray(o.L[o.tet_nodes[v, t]])
        Mp = {}
        for s in (+1, -1):
            m = np.zeros(4)
            Mp[s] = np.zeros(10)
            geo.host_side_moments(_ptr(Lv), s, vol, _ptr(m), _ptr(Mp[s]))
        dsc = np.ascontiguousarray(o.Dinvsqrt[o.enr_id[o.tet_nodes[v, t]]])
        sv = sc.ravel()[v]
        lame = np.array([lp[0] * sv, lp[1] * sv, lm[0] * sv, lm[1] * sv])
        K = np.zeros(300)
        geo.host_cut_element_matrix(_ptr(Lv), int(t), _ptr(np.ascontiguousarray(o.h)), _ptr(Mp[+1]),
                                    _ptr(Mp[-1]), _ptr(dsc), _ptr(lame), _ptr(K))
        _, Ko, _ = o.cut_element(idx)
        worst = max(worst, np.abs(K - Ko[iu]).max() / np.abs(Ko).max())
    assert worst < 1e-13, worst


def test_scaling_and_block_inverse_match_the_oracle(geo):
    """D0 per enriched DOF (eq. XFFT_diagonal) and the off-diagonal entries of the per-node
    enriched Gram blocks, summed from the per-tet terms of the CUDA path, against the oracle's
    quadrature; the 3 x 3 inverse of each scaled block against numpy's inverse."""
    n = (8, 10, 6)
    ell = (1.1, 0.9, 1.0)
    L = synth.sphere_levelset(n, (0.5, 0.45, 0.55), 0.3, ell)
    o = XFEM(L, n, ell)
    vol = float(np.prod(o.h)) / 6.0
    D = np.zeros((o.nX, 3))
    off = np.zeros((o.nX, 3))
    for v, t in o.cut_list:
        Lv = np.ascontiguousarray(o.L[o.tet_nodes[v, t]])
        Mp = {}
        for s in (+1, -1):
            m = np.zeros(4)
            Mp[s] = np.zeros(10)
            geo.host_side_moments(_ptr(Lv), s, vol, _ptr(m), _ptr(Mp[s]))
        acc = np.zeros(12)
        of = np.zeros(12)
        geo.host_cut_scaling(_ptr(Lv), int(t), _ptr(np.ascontiguousarray(o.h)), _ptr(Mp[+1]), _ptr(Mp[-1]),
                             _ptr(acc), _ptr(of))
        eids = o.enr_id[o.tet_nodes[v, t]]
        np.add.at(D, eids, acc.reshape(4, 3))
        np.add.at(off, eids, of.reshape(4, 3))
    assert np.abs(D - o.D).max() < 1e-12 * np.abs(o.D).max()
    ref_off = np.stack([o.Dblk[:, 0, 1], o.Dblk[:, 0, 2], o.Dblk[:, 1, 2]], axis=1)
    assert np.abs(off - ref_off).max() < 1e-12 * np.abs(o.D).max()
    worst = 0.0
    for j in range(o.nX):
        B = o.Bblk[j]
        a = np.array([B[0, 0], B[1, 1], B[2, 2], B[1, 0], B[2, 0], B[2, 1]])
        inv = np.zeros(6)
        assert geo.host_block_inverse(_ptr(a), _ptr(inv)) == 1
        R = np.linalg.inv(B)
        worst = max(worst, np.abs(inv - [R[0, 0], R[1, 1], R[2, 2], R[1, 0], R[2, 0], R[2, 1]]).max()
                    / np.abs(R).max())
    assert worst < 1e-12, worst
    # a non-positive-definite block is refused and leaves the identity
    inv = np.zeros(6)
    assert geo.host_block_inverse(_ptr(np.array([1.0, 1.0, 1.0, 2.0, 0.0, 0.0])), _ptr(inv)) == 0
    assert np.array_equal(inv, [1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
