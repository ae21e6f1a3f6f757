"""ctypes binding of libxfft (include/xfft.h): argument marshalling only.

Every computation runs in the CUDA library; if ``libxfft.so`` cannot be loaded the import of
:func:`lib` raises, there is no fallback.  Arrays may be NumPy arrays (host memory) or torch
CUDA tensors (device memory); one call uses one kind for all of its arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxfft.so")

XFFT_OK, XFFT_EINVAL, XFFT_ENOMEM, XFFT_ECUDA, XFFT_ENOTCONV, XFFT_EBREAKDOWN, XFFT_ETIMEOUT, \
    XFFT_EUNSUPPORTED, XFFT_ESTATE = range(9)
XFFT_FP64, XFFT_FP32_REFINED, XFFT_DW = 0, 1, 2
BB_RULES = {"bb1": 0, "bb2": 1, "alt": 2, "bb1e": 3, "bb2e": 4}
_PREC = {"fp64": XFFT_FP64, "fp32": XFFT_FP32_REFINED, "dw": XFFT_DW}

EXPORTED = (
    "xfft_default_options", "xfft_create", "xfft_set_microstructure",
    "xfft_set_microstructure_phases", "xfft_solve",
    "xfft_effective_stiffness", "xfft_grad", "xfft_grad_phases", "xfft_apply", "xfft_precondition", "xfft_get_setup",
    "xfft_num_enriched", "xfft_num_cut_tets", "xfft_status_string", "xfft_last_error",
    "xfft_destroy", "xfft_profile", "xfft_profile_read", "xfft_apply_noalloc",
    "xfft_batch_effective_stiffness", "xfft_get_tuning", "xfft_fma_rate",
)
NOALLOC_MAX_RHS = 8
PROF_KINDS = ("apply_uncut_f32", "apply_cut_f32", "apply_uncut_f64", "apply_cut_f64", "prec_f32",
              "prec_f64", "vector", "finalize", "setup", "grad", "post", "apply_uncut_dw",
              "apply_cut_dw")


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("len", C.c_double * 3)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("maxit", C.c_int),
                ("snap_tau", C.c_double), ("enr_precond", C.c_int), ("inner_tol", C.c_double),
                ("max_refine", C.c_int), ("poll_every", C.c_int), ("scheme", C.c_int),
                ("step", C.c_double), ("cut_cache", C.c_int), ("bb_rule", C.c_int),
                ("bb_cycle", C.c_int), ("enrichment", C.c_int), ("max_device_bytes", C.c_longlong),
                ("spin_limit_ns", C.c_longlong), ("autotune", C.c_int), ("residual_update", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_rhs", C.c_int), ("iters", C.c_int * 64), ("final_res", C.c_double * 64),
                ("refine_steps", C.c_int), ("n_fe", C.c_int), ("n_x", C.c_int),
                ("n_cut_tets", C.c_int), ("ms_setup", C.c_double), ("ms_solve", C.c_double)]

    def to_dict(self):
        k = self.n_rhs
        return {"iters": list(self.iters[:k]), "final_res": list(self.final_res[:k]),
                "refine_steps": self.refine_steps, "n_fe": self.n_fe, "n_x": self.n_x,
                "n_cut_tets": self.n_cut_tets, "ms_setup": self.ms_setup, "ms_solve": self.ms_solve}


_lib = None


def lib():
    """Load libxfft.so (raises OSError/RuntimeError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libxfft.so is not built; run paper_2601_02172_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.xfft_default_options.argtypes = [C.POINTER(Options)]
    L.xfft_create.argtypes = [C.POINTER(vp), C.POINTER(Grid), C.POINTER(Options), vp]
    L.xfft_set_microstructure.argtypes = [vp, vp, C.POINTER(d), C.POINTER(d), vp, i]
    L.xfft_set_microstructure_phases.argtypes = [vp, i, vp, C.POINTER(d), vp, i]
    L.xfft_solve.argtypes = [vp, i, C.POINTER(d), vp, vp, vp, C.POINTER(d), C.POINTER(Stats), i]
    L.xfft_effective_stiffness.argtypes = [vp, C.POINTER(d), C.POINTER(Stats)]
    L.xfft_grad.argtypes = [vp, C.POINTER(d), C.POINTER(d), vp, C.POINTER(d), i]
    L.xfft_grad_phases.argtypes = [vp, C.POINTER(d), C.POINTER(d), vp, C.POINTER(d), i]
    L.xfft_apply.argtypes = [vp, i, vp, C.POINTER(d), vp, C.POINTER(d), i, i]
    L.xfft_precondition.argtypes = [vp, i, vp, vp, C.POINTER(d), i, i]
    L.xfft_get_setup.argtypes = [vp, vp, vp, vp]
    L.xfft_num_enriched.argtypes = [vp]
    L.xfft_num_cut_tets.argtypes = [vp]
    L.xfft_status_string.argtypes = [i]
    L.xfft_status_string.restype = C.c_char_p
    L.xfft_last_error.restype = C.c_char_p
    L.xfft_destroy.argtypes = [vp]
    L.xfft_destroy.restype = None
    L.xfft_profile.argtypes = [vp, i]
    L.xfft_profile_read.argtypes = [vp, vp, vp, vp]
    L.xfft_apply_noalloc.argtypes = [vp, i, vp, vp, vp]
    L.xfft_batch_effective_stiffness.argtypes = [i, vp, C.POINTER(d), C.POINTER(Stats)]
    L.xfft_get_tuning.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
    L.xfft_fma_rate.argtypes = [i, C.POINTER(d), vp]
    for name in ("xfft_default_options", "xfft_create", "xfft_set_microstructure",
                 "xfft_set_microstructure_phases", "xfft_solve",
                 "xfft_effective_stiffness", "xfft_grad", "xfft_grad_phases", "xfft_apply", "xfft_precondition",
                 "xfft_get_setup", "xfft_num_enriched", "xfft_num_cut_tets", "xfft_profile",
                 "xfft_profile_read", "xfft_apply_noalloc", "xfft_batch_effective_stiffness",
                 "xfft_get_tuning", "xfft_fma_rate"):
        getattr(L, name).restype = i
    _lib = L
    return L


class XfftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (lib().xfft_status_string(status).decode(), msg))
        self.status = status


def check(status, allow=()):
    if status != XFFT_OK and status not in allow:
        raise XfftError(status, lib().xfft_last_error().decode())
    return status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """Pointer of a contiguous array of the given NumPy dtype (host) or torch CUDA tensor."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError("tensor must be contiguous %s" % want)
        return C.c_void_p(x.data_ptr()), bool(x.is_cuda)
    if not (isinstance(x, np.ndarray) and x.dtype == dtype and x.flags.c_contiguous):
        raise TypeError("array must be a C-contiguous %s ndarray" % np.dtype(dtype).name)
    return C.c_void_p(x.ctypes.data), False


def _dvec(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _ordered(method):
    """Order a library call after the caller's pending work on torch's current stream, and the
    caller's later work after the call (the library runs on the solver's own stream)."""
    import functools

    @functools.wraps(method)
    def wrapper(self, *args, **kwargs):
        ts = self._tstream
        if ts is None:
            return method(self, *args, **kwargs)
        import torch
        cur = torch.cuda.current_stream()
        ts.wait_stream(cur)
        out = method(self, *args, **kwargs)
        cur.wait_stream(ts)
        return out
    return wrapper


def check_noalloc_args(stride, device_index, d, q, dAd_sig=None):
    """Shapes and devices of the tensors of ``Solver.apply_noalloc``, checked before anything is
    launched: the library reads d and writes q and dAd_sig through raw pointers sized by the
    number of rows k and the DOF stride, so a short or misplaced tensor would be accessed out of
    bounds on the GPU."""
    ts = (d, q) + (() if dAd_sig is None else (dAd_sig,))
    if not all(_is_torch(x) for x in ts):
        raise TypeError("apply_noalloc takes torch CUDA tensors only")
    if d.dim() != 2 or int(d.shape[1]) != int(stride) or int(d.shape[0]) < 1:
        raise ValueError("d must be (k, %d) with k >= 1" % stride)
    if tuple(q.shape) != tuple(d.shape):
        raise ValueError("q must have the shape of d")
    if dAd_sig is not None and tuple(dAd_sig.shape) != (int(d.shape[0]), 7):
        raise ValueError("dAd_sig must be (k, 7)")
    import torch
    for x in ts:
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("apply_noalloc takes contiguous float64 tensors")
        if not x.is_cuda or x.device.index != device_index:
            raise ValueError("tensors must be on the solver's device cuda:%d" % device_index)


class Solver:
    """One grid on the current CUDA device (thin wrapper of ``xfft_ctx``).

    stream: None (default) gives the solver its own CUDA stream (ordered against torch's current
    stream at every call; the CG iterations then replay as captured CUDA graphs), "legacy" the
    legacy default stream, or a ``torch.cuda.Stream`` / raw ``cudaStream_t`` handle.
    """

    def __init__(self, n, length=(1.0, 1.0, 1.0), precision="fp64", tol=1e-10, maxit=10000,
                 snap_tau=0.0, inner_tol=1e-5, max_refine=20, poll_every=8, stream=None,
                 enr_precond="identity", scheme="cg", step=0.0, cut_cache=False, bb_rule="bb1",
                 bb_cycle=1, enrichment=True, max_device_bytes=0, spin_limit_ns=-1, autotune=True,
                 residual_update=True):
        L = lib()
        self.n = tuple(int(v) for v in n)
        self.length = tuple(float(v) for v in length)
        self.N = int(np.prod(self.n))
        g = Grid()
        for a in range(3):
            g.n[a] = self.n[a]
            g.len[a] = self.length[a]
        o = Options()
        L.xfft_default_options(C.byref(o))
        o.precision = XFFT_FP64 if precision == "fp64" else XFFT_FP32_REFINED
        o.tol = tol
        o.maxit = maxit
        o.snap_tau = snap_tau
        o.inner_tol = inner_tol
        o.max_refine = max_refine
        o.poll_every = poll_every
        o.enr_precond = {"identity": 0, "block3": 1}[enr_precond]
        o.scheme = {"cg": 0, "basic": 1, "bb": 2, "nlcg": 3}[scheme]
        o.step = step
        o.cut_cache = int(bool(cut_cache))
        o.bb_rule = BB_RULES[bb_rule]
        o.bb_cycle = int(bb_cycle)
        o.enrichment = int(bool(enrichment))
        o.max_device_bytes = int(max_device_bytes)
        o.spin_limit_ns = int(spin_limit_ns)
        o.autotune = int(bool(autotune))
        o.residual_update = int(bool(residual_update))
        self.precision = precision
        self.num_phases = 0
        try:
            import torch
            self.device_index = torch.cuda.current_device() if torch.cuda.is_available() else -1
        except ImportError:
            self.device_index = -1
        self._ctx = C.c_void_p()
        self._tstream = None
        handle = None
        if stream is None or _is_torch(stream):
            import torch
            if stream is None:
                stream = torch.cuda.Stream()
            self._tstream = stream
            handle = stream.cuda_stream
        elif stream != "legacy":
            handle = int(stream)
        check(L.xfft_create(C.byref(self._ctx), C.byref(g), C.byref(o),
                            C.c_void_p(handle) if handle else None))

    def close(self):
        if self._ctx:
            lib().xfft_destroy(self._ctx)
            self._ctx = C.c_void_p()

    __del__ = close

    @property
    def num_enriched(self):
        return lib().xfft_num_enriched(self._ctx)

    @property
    def num_cut_tets(self):
        return lib().xfft_num_cut_tets(self._ctx)

    @property
    def tuning(self):
        """(cut-tet kernel grid in blocks, its right-hand sides per launch, the preconditioner's
        right-hand sides per group of FFT passes) in use."""
        b, r, g = C.c_int(), C.c_int(), C.c_int()
        check(lib().xfft_get_tuning(self._ctx, C.byref(b), C.byref(r), C.byref(g)))
        return b.value, r.value, g.value

    @property
    def stride(self):
        return 3 * (self.N + self.num_enriched)

    @_ordered
    def set_microstructure(self, L, lame_minus, lame_plus, scale=None):
        Lp, dev = _ptr(L, np.float64)
        sp_, sdev = _ptr(scale, np.float32)
        if scale is not None and sdev != dev:
            raise TypeError("L and scale must both be host or both be device arrays")
        lm, lmp = _dvec(lame_minus)
        lp, lpp = _dvec(lame_plus)
        check(lib().xfft_set_microstructure(self._ctx, Lp, lmp, lpp, sp_, int(dev)))
        self.num_phases = 2

    @_ordered
    def set_microstructure_phases(self, Ls, phases, scale=None):
        """Several interfaces: ``Ls`` holds K nodal level sets (shape (K,) + n), ``phases`` the
        K + 1 pairs (lambda, mu); a point lies in phase k if L_k is the first negative level
        set there, in phase K if none is (see ``xfft_set_microstructure_phases``)."""
        Lp, dev = _ptr(Ls, np.float64)
        sp_, sdev = _ptr(scale, np.float32)
        if scale is not None and sdev != dev:
            raise TypeError("Ls and scale must both be host or both be device arrays")
        K = int(Ls.shape[0]) if Ls.ndim == 4 else 1
        if int(np.prod(Ls.shape)) != K * self.N:
            raise ValueError("Ls must hold K level sets of the grid's N nodes")
        lame, lp = _dvec(np.asarray(phases, dtype=np.float64).reshape(-1))
        if lame.size != 2 * (K + 1):
            raise ValueError("K level sets need K + 1 phases (lambda, mu)")
        check(lib().xfft_set_microstructure_phases(self._ctx, K, Lp, lp, sp_, int(dev)))
        self.num_phases = K + 1

    @_ordered
    def solve(self, eps, u=True, voxel_stress=False, device=None):
        """Solve for the Mandel strains ``eps`` (k x 6).  Host (NumPy) outputs unless
        ``device`` is a torch device, in which case outputs are CUDA tensors."""
        e, ep = _dvec(np.atleast_2d(eps))
        k = e.shape[0]
        nX = self.num_enriched
        out = {}
        if device is not None:
            import torch
            us = torch.empty((k, 3, self.N), dtype=torch.float64, device=device) if u else None
            ue = torch.empty((k, 3, max(nX, 1)), dtype=torch.float64, device=device) if u else None
            vs = torch.empty((k, 6, self.N), dtype=torch.float64, device=device) if voxel_stress else None
            dev = 1
        else:
            us = np.empty((k, 3, self.N)) if u else None
            ue = np.empty((k, 3, max(nX, 1))) if u else None
            vs = np.empty((k, 6, self.N)) if voxel_stress else None
            dev = 0
        ms = np.empty((k, 6))
        st = Stats()
        status = check(lib().xfft_solve(self._ctx, k, ep, _ptr(us, np.float64)[0],
                                        _ptr(ue, np.float64)[0], _ptr(vs, np.float64)[0],
                                        ms.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st), dev),
                       allow=(XFFT_ENOTCONV,))
        out["u_std"] = us
        out["u_enr"] = ue[:, :, :nX] if ue is not None else None
        out["voxel_stress"] = vs
        out["mean_stress"] = ms
        out["stats"] = st.to_dict()
        out["converged"] = status == XFFT_OK
        return out

    @_ordered
    def effective_stiffness(self):
        Cm = np.empty(36)
        st = Stats()
        status = check(lib().xfft_effective_stiffness(self._ctx, Cm.ctypes.data_as(C.POINTER(C.c_double)),
                                                      C.byref(st)), allow=(XFFT_ENOTCONV,))
        return Cm.reshape(6, 6), dict(st.to_dict(), converged=status == XFFT_OK)

    @_ordered
    def grad(self, G, scale_grad=True, device=None):
        """dLoss/d(lam-, mu-, lam+, mu+) (several interfaces: lam_0, mu_0, lam_1, mu_1, ...),
        dLoss/ds_v (float32) and the energy-form C_eff for G = dLoss/dC_eff of the last
        effective_stiffness call."""
        g, gp = _dvec(np.asarray(G, dtype=np.float64).reshape(36))
        dl = np.empty(2 * max(self.num_phases, 2))
        ce = np.empty(36)
        if scale_grad:
            if device is not None:
                import torch
                ds = torch.empty(self.N, dtype=torch.float32, device=device)
            else:
                ds = np.empty(self.N, dtype=np.float32)
        else:
            ds = None
        dsp, dev = _ptr(ds, np.float32)
        check(lib().xfft_grad_phases(self._ctx, gp, dl.ctypes.data_as(C.POINTER(C.c_double)), dsp,
                              ce.ctypes.data_as(C.POINTER(C.c_double)), int(bool(dev))))
        return dl, ds, ce.reshape(6, 6)

    @_ordered
    def apply(self, d, eps=None, precision="fp64", stress=True):
        """q = A d (+ b(eps)) on full DOF vectors (k x stride, scaled enriched part).
        precision: "fp64", "fp32" or "dw" (double-word kernels on FP64 data).  stress=False
        (without eps) skips the stress integrals (sig is None): with "fp32" these are the
        kernels of the FP32 CG iterations."""
        d = np.ascontiguousarray(np.atleast_2d(d), dtype=np.float64)
        k = d.shape[0]
        q = np.empty_like(d)
        sig = np.empty((k, 6)) if (stress or eps is not None) else None
        if eps is not None:
            e, ep = _dvec(np.atleast_2d(eps))
        else:
            ep = None
        check(lib().xfft_apply(self._ctx, k, C.c_void_p(d.ctypes.data), ep, C.c_void_p(q.ctypes.data),
                               sig.ctypes.data_as(C.POINTER(C.c_double)) if sig is not None else None,
                               _PREC[precision], 0))
        return q, sig

    @_ordered
    def apply_noalloc(self, d, q, dAd_sig=None):
        """Allocation-free FP64 apply on caller-owned CUDA tensors (k x stride): q = A d; if
        given, dAd_sig (k x 7) receives <d, A d> and int_Y C grad^s d.  The library allocates
        nothing in this call."""
        check_noalloc_args(self.stride, self.device_index, d, q, dAd_sig)
        k = int(d.shape[0])
        dp, _ = _ptr(d, np.float64)
        qp, _ = _ptr(q, np.float64)
        sp_, _ = _ptr(dAd_sig, np.float64)
        check(lib().xfft_apply_noalloc(self._ctx, k, dp, qp, sp_))


    @_ordered
    def precondition(self, f, precision="fp64"):
        f = np.ascontiguousarray(np.atleast_2d(f), dtype=np.float64)
        k = f.shape[0]
        z = np.empty_like(f)
        rr = np.empty(k)
        check(lib().xfft_precondition(self._ctx, k, C.c_void_p(f.ctypes.data), C.c_void_p(z.ctypes.data),
                                      rr.ctypes.data_as(C.POINTER(C.c_double)),
                                      0 if precision == "fp64" else 1, 0))
        return z, rr

    def profile(self, enable=True):
        """Enable (and reset) or disable the library's per-kernel-group event timing."""
        check(lib().xfft_profile(self._ctx, int(bool(enable))))

    @_ordered
    def profile_read(self):
        """{group: (ms, launches, rhs_units)} accumulated since profile(True)."""
        ms = np.zeros(16)
        la = np.zeros(16, dtype=np.int64)
        un = np.zeros(16, dtype=np.int64)
        check(lib().xfft_profile_read(self._ctx, C.c_void_p(ms.ctypes.data), C.c_void_p(la.ctypes.data),
                                      C.c_void_p(un.ctypes.data)))
        return {k: (float(ms[i]), int(la[i]), int(un[i])) for i, k in enumerate(PROF_KINDS)}

    @_ordered
    def setup_info(self):
        nX = self.num_enriched
        en = np.empty(max(nX, 1), dtype=np.int32)
        D0 = np.empty((max(nX, 1), 3))
        code = np.empty(self.N, dtype=np.uint16)
        check(lib().xfft_get_setup(self._ctx, C.c_void_p(en.ctypes.data), C.c_void_p(D0.ctypes.data),
                                   C.c_void_p(code.ctypes.data)))
        return en[:nX], D0[:nX], code


def fma_rate(precision="fp64"):
    """Measured FMA throughput (FLOP/s) of the current GPU in FP64 ("fp64") or FP32 ("fp32")."""
    r = C.c_double()
    check(lib().xfft_fma_rate(XFFT_FP64 if precision == "fp64" else XFFT_FP32_REFINED, C.byref(r), None))
    return r.value


def batch_effective_stiffness(solvers):
    """C_eff (list of 6x6) and stats of several solvers at once (``xfft_batch_effective_stiffness``:
    the solvers advance in lockstep and every inner CG solve of all of them runs as one
    device-driven graph launch)."""
    import torch
    n = len(solvers)
    arr = (C.c_void_p * n)(*[sv._ctx for sv in solvers])
    Cm = np.empty((n, 36))
    st = (Stats * n)()
    cur = torch.cuda.current_stream()
    for sv in solvers:
        if sv._tstream is not None:
            sv._tstream.wait_stream(cur)
    status = lib().xfft_batch_effective_stiffness(n, arr, Cm.ctypes.data_as(C.POINTER(C.c_double)), st)
    for sv in solvers:
        if sv._tstream is not None:
            cur.wait_stream(sv._tstream)
    check(status, allow=(XFFT_ENOTCONV,))
    return [Cm[i].reshape(6, 6) for i in range(n)], [st[i].to_dict() for i in range(n)]
