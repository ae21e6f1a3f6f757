"""The CUDA path's per-frequency Green solve, compiled for the host (no GPU), against the oracle.

`csrc/fft_fast.cuh` factorises M(xi) = Z(xi)^H A0_v Z(xi) (eq. GreenHermitian) in closed form
from the per-axis phase factors e_a = exp(i theta_a), s_a = e_a - 1 (theta_a = 2 pi k_a / n_a,
the tables the library builds) and solves M x = F by two triangular solves.  Here it is built
into a host library and compared with a dense solve of the oracle's symbol, which the oracle
forms from the assembled voxel reference matrix, at every frequency of an anisotropic grid.
The radix butterflies of the same file's Stockham stages are checked against direct DFTs.
"""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import XFEM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

pytestmark = pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")


@pytest.fixture(scope="module")
def green(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("hostgreen") / "libgreen.so")
    src = os.path.join(ROOT, "tests", "host", "green_host.cu")
    inc = ["-I" + os.path.join(ROOT, "paper_2601_02172_gb300", "csrc"), "-I" + os.path.join(ROOT, "include")]
    subprocess.run([NVCC, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC"]
                   + inc + ["-o", out, src], check=True, capture_output=True)
    lib = C.CDLL(out)
    dp = C.POINTER(C.c_double)
    lib.host_green_solve.argtypes = [C.c_int, dp, dp, dp, C.c_double, dp]
    lib.host_green_solve.restype = C.c_int
    return lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


@pytest.mark.parametrize("dbl,tol", [(1, 1e-12), (0, 2e-5)])
def test_green_solve_matches_the_oracle_symbol(green, dbl, tol):
    n = (6, 8, 10)
    ell = (1.2, 0.9, 1.1)
    o = XFEM(synth.sphere_levelset(n, (0.5, 0.5, 0.5), 0.3, ell), n, ell)
    h = [ell[a] / n[a] for a in range(3)]
    ih = np.array([1.0 / x for x in h])
    halfvol = 0.5 * h[0] * h[1] * h[2] / 6.0
    rng = np.random.default_rng(5)
    worst = 0.0
    for k in np.ndindex(*n):
        e = np.zeros(6)
        s = np.zeros(6)
        for a in range(3):
            th = 2.0 * math.pi * k[a] / n[a]
            e[2 * a:2 * a + 2] = (math.cos(th), math.sin(th))
            s[2 * a:2 * a + 2] = (-2.0 * math.sin(0.5 * th) ** 2, math.sin(th))
        Fc = rng.normal(size=3) + 1j * rng.normal(size=3)
        F = np.column_stack([Fc.real, Fc.imag]).ravel().copy()
        ok = green.host_green_solve(dbl, _p(e), _p(s), _p(ih), halfvol, _p(F))
        if k == (0, 0, 0):
            assert ok == 0  # the mean maps to zero
            continue
        assert ok == 1, k
        x = F[0::2] + 1j * F[1::2]
        ref = np.linalg.solve(o.green_symbol_at(k), Fc)
        worst = max(worst, np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert worst < tol, worst


@pytest.fixture(scope="module")
def dft(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("hostdft") / "libdft.so")
    src = os.path.join(ROOT, "tests", "host", "dft_host.cu")
    inc = ["-I" + os.path.join(ROOT, "paper_2601_02172_gb300", "csrc"), "-I" + os.path.join(ROOT, "include")]
    subprocess.run([NVCC, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-shared", "-Xcompiler", "-fPIC"]
                   + inc + ["-o", out, src], check=True, capture_output=True)
    lib = C.CDLL(out)
    lib.host_dft.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.host_dft.restype = C.c_int
    return lib


@pytest.mark.parametrize("R", [2, 3, 4, 5, 6, 8, 16])
@pytest.mark.parametrize("inv", [0, 1])
def test_radix_butterflies_are_dfts(dft, R, inv):
    """Each radix-R butterfly of the FFT stages is the length-R DFT, exp(-2 pi i jk/R)
    forward and exp(+2 pi i jk/R) inverse (unnormalised)."""
    rng = np.random.default_rng(R + 10 * inv)
    x = rng.normal(size=R) + 1j * rng.normal(size=R)
    v = np.column_stack([x.real, x.imag]).ravel().copy()
    assert dft.host_dft(R, inv, _p(v)) == 1
    y = v[0::2] + 1j * v[1::2]
    jk = np.outer(np.arange(R), np.arange(R))
    ref = np.exp((2j if inv else -2j) * np.pi * jk / R) @ x
    assert np.abs(y - ref).max() < 1e-14 * max(1.0, np.abs(ref).max())
