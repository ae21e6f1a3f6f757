#!/usr/bin/env python3
"""Benchmark of the X-FFT hot path on GB300.

One step = the whole hot path for one microstructure: GPU setup of the 128^3 X-FEM
discretization (snap, classification, enriched numbering, cut-tet moments, scaling), the six
unit load cases solved as one batch by FP32 PCG with FP64 residual refinement, the effective
stiffness, and the adjoint gradient of ||C_eff - C_target||_F^2 with respect to the four phase
Lame constants and the per-voxel modulus scale.  Inputs are resident in HBM when the timed region
starts (``value``); ``e2e`` repeats the step through the C-ABI with host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xfft|reference]
Multi-GPU runs (torchrun) are replicas: every rank solves its own copy of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "X-FFT solves/s (6 load cases) & DOF-iters/s at 128^3, %HBM roofline, FP32 vs FP64"
UNIT = "solves/s"
WORKLOAD = ("ellipsoids40: 128^3 periodic grid, 40 random ellipsoids (aspect 1-3, random "
            "orientation, vf 25%), contrast E_incl/E_matrix = 50 (nu 0.2/0.3), per-voxel modulus "
            "scale U[0.8,1.2]; six unit Mandel load cases; loss ||C_eff - C_target||_F^2")

# algorithmic bytes per launch and per processed right-hand side of the timed kernel groups
def algorithmic_bytes(kind, N, nX, ncut, has_scale, cut_cache=False):
    """Algorithmic bytes of one kernel group as (per launch, per right-hand side)."""
    geo = N * (2 + (4 if has_scale else 0))
    if kind == "apply_cut_f32" and cut_cache:
        # cached element matrices: per launch each cut tet's packed matrix (1200 B) and node and
        # enriched ids (32 B); per RHS the DOFs of the enriched nodes (all nodes of cut tets):
        # std and enr d read (24 B) and std and enr q atomically updated (48 B)
        return 1232 * ncut, 72 * nX
    if kind in ("apply_cut_f32", "apply_cut_f64"):
        return cut_bytes(kind[-3:], nX, ncut)
    per = _per_rhs_bytes(kind, N, nX, ncut, geo)
    return (0, per) if per is not None else None


def _per_rhs_bytes(kind, N, nX, ncut, geo):
    if kind == "apply_uncut_f32":  # the fused CG form: z, d_old, u in; d_new, u, q out
        return 72 * N + geo
    if kind == "apply_uncut_f64":
        return 48 * N + geo
    if kind == "prec_f32":  # fused form: f, q in; f (f -= alpha q) and z out
        return 48 * (N + nX)
    if kind == "prec_f64":
        return 48 * (N + nX)
    return None


REC_REALS = 68  # reals of a cut tet's apply record (geometry, moduli, 1/sqrt(D0) of its DOFs)
# algorithmic flops of the stencil per voxel and right-hand side: six Kuhn tets of about 35 each
# (gradient columns, trace, stress, edge tensions) and the corner forces
STENCIL_FLOPS = 250


def cut_bytes(prec, nX, ncut):
    """Unique bytes of one cut-tet apply as (per launch, per right-hand side): each cut tet's
    apply record once per launch (68 reals: per-side moments, P = M c, gamma, scaled moduli and
    the 1/sqrt(D0) of its 12 enriched DOFs), its node and enriched ids (8 ints) and tet type (1
    int); per right-hand side, at every enriched node (the nodes of the cut tets), the standard
    and enriched d read (6 reals) and q updated (6 reals read and written): 72 B in FP32, 144 B
    in FP64."""
    r = 4 if prec == "f32" else 8
    return (36 + REC_REALS * r) * ncut, 18 * r * nX


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("xfft", "reference"), default="xfft")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the block-preconditioner, batch and cuFFT side measurements")
    ap.add_argument("--cpu-n", type=int, default=16)
    ap.add_argument("--cut-cache", action="store_true",
                    help="run the timed solves with the cached cut-tet element matrices")
    ap.add_argument("--enr", choices=("block3", "identity"), default="block3",
                    help="preconditioner on the enriched DOFs: the 3x3 node blocks (default) or the "
                         "paper's identity; the other one is timed beside it")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_case(job):
    """One load case of the CPU oracle's PCG (FFT Green operator), run in a worker process."""
    o, k, tol = job
    e = np.eye(6)[k]
    t0 = time.perf_counter()
    u, info = o.pcg(e, tol=tol, green="fft")
    return k, time.perf_counter() - t0, int(info["iters"]), o.mean_stress(u, e)


def resampled_workload(n_cpu, name="ellipsoids40"):
    """The bench workload's ellipsoids (and scale field, subsampled) on an n_cpu^3 grid; or, for
    name "single_sphere", the 16^3 single-sphere case (no scale field)."""
    import synth
    if name == "single_sphere":
        w = synth.make_workload("single_sphere")
        return w["L"], None, w["lame_minus"], w["lame_plus"]
    w = synth.make_workload("ellipsoids40")
    n = (n_cpu,) * 3
    L = synth.ellipsoids_levelset(n, w["info"]["inclusions"])
    step = 128 // n_cpu if 128 % n_cpu == 0 else 1
    sc = np.ascontiguousarray(w["scale"][::step, ::step, ::step][:n_cpu, :n_cpu, :n_cpu]).astype(np.float32)
    return L, sc, w["lame_minus"], w["lame_plus"]


def oracle_pool(workers):
    """Worker processes for the oracle's six load cases (spawned: safe after CUDA is initialised)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def oracle_solve(n_cpu, tol, pool, name="ellipsoids40"):
    """The CPU oracle as it stands, one whole six-case solve of the resampled workload: setup and
    assembly in this process, then the six load cases' PCG spread over the worker pool (they
    are independent).  Returns times, iteration counts and C_eff."""
    from oracle import XFEM
    L, sc, lm, lp = resampled_workload(n_cpu, name)
    t0 = time.perf_counter()
    o = XFEM(L, (n_cpu,) * 3, lame_minus=lm, lame_plus=lp, scale=sc)
    o.assemble()
    t1 = time.perf_counter()
    res = pool.map(_oracle_case, [(o, k, tol) for k in range(6)])
    t2 = time.perf_counter()
    C = np.zeros((6, 6))
    for k, _, _, sig in res:
        C[:, k] = sig
    iters = [r[2] for r in res]
    return {"n": n_cpu, "ncut": len(o.cut_list), "ndof": o.ndof, "t_setup": t1 - t0,
            "t_pcg": t2 - t1, "t": t2 - t0, "iters": iters, "C": C,
            "dofit": o.ndof * sum(iters) / (t2 - t1)}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def _sample_text(r, tol, workers):
    return ("ellipsoids40 resampled at %d^3 (%d cut tets, %d DOF): the oracle's whole six-case "
            "solve, tol %g, measured (not scaled): setup + assembly %.1f s on 1 core, six PCGs "
            "(%s iterations) %.1f s on %d worker processes" % (
                r["n"], r["ncut"], r["ndof"], tol, r["t_setup"],
                "/".join(str(i) for i in r["iters"]), r["t_pcg"], workers))


def _gpu_same_input(n_cpu, tol, r, name="ellipsoids40"):
    """The GPU's set-up + six-case solve of the oracle's input (host level set), same tolerance."""
    import torch
    from paper_2601_02172_gb300 import Solver
    L, sc, lm, lp = resampled_workload(n_cpu, name)
    same = {}
    for prec in ("fp64", "fp32"):
        sv = Solver((n_cpu,) * 3, precision=prec, tol=tol)
        sv.set_microstructure(L, lm, lp, sc)
        sv.effective_stiffness()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 5
        for _ in range(reps):
            sv.set_microstructure(L, lm, lp, sc)
            Cg, _ = sv.effective_stiffness()
        torch.cuda.synchronize()
        same[prec] = {"solves_per_s": reps / (time.perf_counter() - t0),
                      "ceff_rel_diff_vs_oracle": float(np.abs(Cg - r["C"]).max() / np.abs(r["C"]).max())}
        sv.close()
    return same


def cpu_baseline(n_cpu, tol, dev=None, more=True):
    """The oracle timed on this host on the resampled workload, and the GPU on the same input;
    with more, also the 16^3 single sphere (config 1) and the workload resampled at 32^3."""
    workers = min(6, _cores())
    with oracle_pool(workers) as pool:
        r = oracle_solve(n_cpu, tol, pool)
        others = []
        if more:
            for name, nn in (("single_sphere", 16), ("ellipsoids40", 32)):
                others.append((name, nn, oracle_solve(nn, tol, pool, name)))
    out = {"value": 1.0 / r["t"], "unit": UNIT, "cores": workers, "kind": "oracle",
           "sample": _sample_text(r, tol, workers), "dof_iters_per_s": r["dofit"],
           "os_cpu_count": os.cpu_count(), "affinity_cores": _cores()}
    if dev is not None:
        out["gpu_same_input"] = dict(_gpu_same_input(n_cpu, tol, r),
                                     note="the GPU's setup + six-case solve of the identical %d^3 input "
                                          "(host level set), same tolerance" % n_cpu)
        more_out = []
        for name, nn, ro in others:
            more_out.append({"input": "%s at %d^3" % (name, nn), "ncut": ro["ncut"], "ndof": ro["ndof"],
                             "oracle_solves_per_s": 1.0 / ro["t"], "oracle_setup_s": ro["t_setup"],
                             "oracle_pcg_s": ro["t_pcg"], "oracle_iters": ro["iters"],
                             "gpu": _gpu_same_input(nn, tol, ro, name)})
        out["more_samples"] = more_out
    return out


def run_reference(args):
    """Reference arm: the CPU oracle as it stands; each step is one measured six-case solve of the
    workload resampled at --cpu-n^3 (a bounded sample of the 128^3 workload)."""
    workers = min(6, _cores())
    ts, rs = [], []
    with oracle_pool(workers) as pool:
        for k in range(args.warmup + args.steps):
            r = oracle_solve(args.cpu_n, args.tol, pool)
            if k >= args.warmup:
                rs.append(r)
                ts.append(r["t"])
    t = statistics.mean(ts)
    value = 1.0 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "tol": args.tol,
                       "sample": "each step: the oracle's whole six-case solve of the workload "
                                 "resampled at %d^3, measured" % args.cpu_n},
            "cpu_baseline": {"kind": "oracle", "cores": workers, "value": value, "unit": UNIT,
                             "sample": _sample_text(rs[-1], args.tol, workers),
                             "dof_iters_per_s": statistics.mean(r["dofit"] for r in rs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def traffic_for(kind):
    """DRAM bytes per launch and RHS from the committed ncu summary, if the kernel source has
    not changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(kind)
    if not ent:
        return None
    srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
    h = hashlib.sha256()
    for f in srcs:
        p = os.path.join(ROOT, "paper_2601_02172_gb300", "csrc", f)
        if not os.path.exists(p):
            return None
        h.update(open(p, "rb").read())
    sha = h.hexdigest()[:16]
    if sha != ent.get("source_sha"):
        return None
    return ent


def max_over_ranks(ms, dist, device):
    """The slowest rank's time of the timed region (every rank gets it)."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, ms):
    """Whole-job rate: every replica solved `steps` six-case problems in `ms` (the max over ranks)."""
    return world * steps / (ms / 1000.0)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    import synth
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_02172_gb300 import Solver

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = (args.n,) * 3
    w = synth.make_workload("ellipsoids40", n=n)
    N = int(np.prod(n))
    lm, lp = w["lame_minus"], w["lame_plus"]
    L_h = np.ascontiguousarray(w["L"])
    s_h = np.ascontiguousarray(w["scale"])
    L_d = torch.from_numpy(L_h).to(dev)
    s_d = torch.from_numpy(s_h).to(dev)
    L_pin = torch.from_numpy(L_h).pin_memory()  # e2e inputs come from pinned host memory
    s_pin = torch.from_numpy(s_h).pin_memory()
    solver = Solver(n, precision="fp32", tol=args.tol, cut_cache=args.cut_cache, enr_precond=args.enr)

    # C_target: a random SPD perturbation of C_eff (seeded)
    solver.set_microstructure(L_d, lm, lp, s_d)
    C0, _ = solver.effective_stiffness()
    rng = np.random.default_rng(4)
    while True:
        G = rng.normal(size=(6, 6))
        G = 0.5 * (G + G.T)
        Ct = C0 + 0.05 * np.linalg.norm(C0) / np.linalg.norm(G) * G
        if np.linalg.eigvalsh(Ct).min() > 0:
            break

    info = {"iters": 0, "dofit": 0.0, "ncut": solver.num_cut_tets, "nX": 0}

    def step(device_inputs=True):
        if device_inputs:
            solver.set_microstructure(L_d, lm, lp, s_d)
        else:
            solver.set_microstructure(L_pin, lm, lp, s_pin)
        C, st = solver.effective_stiffness()
        dl, ds, _ = solver.grad(2.0 * (C - Ct), device=dev if device_inputs else None)
        nX = solver.num_enriched
        info["nX"] = nX
        info["iters"] += sum(st["iters"])
        info["dofit"] += 3.0 * (N + nX) * sum(st["iters"])
        info["refine"] = st["refine_steps"]
        return C, dl, ds

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    info.update(iters=0, dofit=0.0)
    # the timed region runs the production path: tracing off, so the CG iterations between two
    # convergence polls replay as captured CUDA graphs
    sampler = ClockSampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        C, dl, ds = step()
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    if dist:
        ms = max_over_ranks(ms, dist, dev)
        dist.barrier()
    steps_iters = info["iters"]
    dofit_rate = info["dofit"] / (ms / 1000.0)
    value = job_value(world, args.steps, ms)
    # per-kernel-group device times (roofline): a separate, untimed pass of the same steps with
    # the library's event tracing on (each group bracketed by events on the solver's stream)
    prof_steps = max(1, min(args.steps, 3))
    solver.profile(True)
    for _ in range(prof_steps):
        step()
    prof = solver.profile_read()
    solver.profile(False)
    torch.cuda.synchronize()

    # live roofline of the dominant kernel group
    peak, peak_kind = load_peaks()
    kinds = ["apply_uncut_f32", "prec_f32", "apply_uncut_f64", "prec_f64", "apply_cut_f32", "apply_cut_f64"]
    dom = max(kinds, key=lambda k: prof[k][0])
    kms, klaunch, kunits = prof[dom]
    nX = info["nX"]
    bpl, bpu = algorithmic_bytes(dom, N, nX, info["ncut"], True, cut_cache=args.cut_cache)
    achieved = (bpl * klaunch + bpu * kunits) / (kms / 1000.0) / 1e9 if kms > 0 else 0.0
    tr = traffic_for(dom + ("_cached" if args.cut_cache and dom == "apply_cut_f32" else ""))
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "bytes_per_launch": bpl,
            "bytes_per_rhs": bpu,
            "launches": klaunch, "rhs_units": kunits, "avg_launch_ms": kms / max(klaunch, 1),
            "traffic": (tr["dram_bytes_per_rhs"] * kunits / max(klaunch, 1)) if tr else None,
            "groups_ms_per_step": {k: round(v[0] / prof_steps, 3) for k, v in prof.items()},
            "profiled_steps": prof_steps}
    # the library's kernels per step (counted by the traced pass) times the timed steps
    gpu_launches = int(sum(v[1] for v in prof.values()) * args.steps // prof_steps)

    line = None
    if rank == 0:
        # end to end: host buffers in, host results out, copies inside the timed region
        torch.cuda.synchronize()
        te = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            C_e, dl_e, ds_e = step(device_inputs=False)
            torch.cuda.synchronize()
            te.append(time.perf_counter() - t0)
        e2e = {"value": 1.0 / statistics.mean(te), "unit": UNIT,
               "h2d_bytes_per_step": int(L_h.nbytes + s_h.nbytes + 36 * 8 * 2),
               "d2h_bytes_per_step": int(N * 4 + 36 * 8 * 3 + 4 * 8)}
        extra = {}
        if not args.no_fp64:
            # plain FP64 for comparison: six cases batched, and one case at a time
            s64 = Solver(n, precision="fp64", tol=args.tol)
            s64.set_microstructure(L_d, lm, lp, s_d)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C64, st64 = s64.effective_stiffness()
            torch.cuda.synchronize()
            t_b = time.perf_counter() - t0
            t0 = time.perf_counter()
            its1 = 0
            for k in range(6):
                out = s64.solve(np.eye(6)[k:k + 1], u=False)
                its1 += out["stats"]["iters"][0]
            torch.cuda.synchronize()
            t_1 = time.perf_counter() - t0
            sref = Solver(n, precision="fp64", tol=1e-10)
            sref.set_microstructure(L_d, lm, lp, s_d)
            Cref, _ = sref.effective_stiffness()
            extra["fp64"] = {"solves_per_s_batched6": 1.0 / t_b, "solves_per_s_single_rhs": 1.0 / t_1,
                             "iters_batched6": sum(st64["iters"]), "iters_single_rhs": its1,
                             "tol": args.tol}
            # the FP64 path against the measured FMA peaks (GB300's FP64 rate is far below FP32's):
            # the FP64 stencil at STENCIL_FLOPS per voxel and right-hand side, traced separately
            from paper_2601_02172_gb300.capi import fma_rate
            peak64, peak32 = fma_rate("fp64"), fma_rate("fp32")
            s64.profile(True)
            s64.effective_stiffness()
            p64 = s64.profile_read()
            s64.profile(False)
            ms_u, la_u, un_u = p64["apply_uncut_f64"]
            fl = STENCIL_FLOPS * N * un_u / (ms_u / 1e3) if ms_u > 0 else 0.0
            by = (48 * N + 6 * N) * un_u / (ms_u / 1e3) if ms_u > 0 else 0.0
            extra["fp64"].update({
                "fma_peak_fp64_tflops_measured": peak64 / 1e12, "fma_peak_fp32_tflops_measured": peak32 / 1e12,
                "stencil_fp64": {"ms_per_launch": ms_u / max(la_u, 1), "achieved_tflops": fl / 1e12,
                                 "frac_of_measured_fp64_fma_peak": fl / peak64,
                                 "achieved_gbs": by / 1e9, "frac_of_measured_hbm": by / 1e9 / load_peaks()[0],
                                 "flops_per_voxel_rhs": STENCIL_FLOPS}})
            extra["accuracy"] = {
                "ceff_rel_err_fp32_refined_vs_fp64_tol1e-10": float(np.abs(C - Cref).max() / np.abs(Cref).max()),
                "ceff_rel_err_fp64_vs_fp64_tol1e-10": float(np.abs(C64 - Cref).max() / np.abs(Cref).max())}
            s64.close()
            sref.close()
        if not args.no_extras:
            # the other enriched preconditioner (3x3 node blocks or the paper's identity): the same
            # whole step (set-up, six-case solve, gradient), timed like the headline
            other = "identity" if args.enr == "block3" else "block3"
            sb = Solver(n, precision="fp32", tol=args.tol, enr_precond=other)
            sb.set_microstructure(L_d, lm, lp, s_d)
            sb.effective_stiffness()
            torch.cuda.synchronize()
            e0b, e1b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0b.record()
            its_b = 0
            for _ in range(args.steps):
                sb.set_microstructure(L_d, lm, lp, s_d)
                Cb, stb = sb.effective_stiffness()
                sb.grad(2.0 * (Cb - Ct), device=dev)
                its_b += sum(stb["iters"])
            e1b.record()
            torch.cuda.synchronize()
            extra["enr_" + other] = {"solves_per_s": args.steps / (e0b.elapsed_time(e1b) / 1e3),
                                     "cg_iters_per_step": its_b / args.steps,
                                     args.enr + "_cg_iters_per_step": steps_iters / args.steps,
                                     args.enr + "_solves_per_s": value,
                                     "ceff_rel_diff": float(np.abs(Cb - C).max() / np.abs(C).max())}
            sb.close()
            # many microstructures at once (16 uneven grids x 6 load cases, FP32-refined to 1e-8):
            # one call, one host thread and stream per microstructure, against the same solvers in turn
            from paper_2601_02172_gb300 import batch_effective_stiffness
            bw = synth.batch_uneven(16, seed=3)
            bsolvers = []
            for wb in bw:
                sv = Solver(wb["n"], precision="fp32", tol=1e-8)
                sv.set_microstructure(wb["L"], wb["lame_minus"], wb["lame_plus"])
                bsolvers.append(sv)
            batch_effective_stiffness(bsolvers)  # warm-up (graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Cbat, bst = batch_effective_stiffness(bsolvers)
            torch.cuda.synchronize()
            t_bat = time.perf_counter() - t0
            t0 = time.perf_counter()
            for sv in bsolvers:
                sv.effective_stiffness()
            torch.cuda.synchronize()
            t_seq = time.perf_counter() - t0
            # per-context concurrency: one host thread per solver (ctypes releases the GIL), each
            # with its own stream and device-driven loops
            import concurrent.futures as cf
            with cf.ThreadPoolExecutor(len(bsolvers)) as ex:
                list(ex.map(lambda sv: sv.effective_stiffness(), bsolvers))  # warm
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                list(ex.map(lambda sv: sv.effective_stiffness(), bsolvers))
                torch.cuda.synchronize()
                t_thr = time.perf_counter() - t0
            # accuracy of the FP32-refined batch against plain FP64 solves of the same members
            errs = []
            for wb, Cb in zip(bw, Cbat):
                s64 = Solver(wb["n"], precision="fp64", tol=1e-8)
                s64.set_microstructure(wb["L"], wb["lame_minus"], wb["lame_plus"])
                C64, _s = s64.effective_stiffness()
                errs.append(float(np.abs(Cb - C64).max() / np.abs(C64).max()))
                s64.close()
            extra["batch16"] = {"microstructures": len(bw), "rhs": 6 * len(bw),
                                "ceff_max_rel_err_vs_fp64": max(errs),
                                "grids": [int(wb["n"][0]) for wb in bw], "tol": 1e-8,
                                "solves_per_s_batched": len(bw) / t_bat,
                                "solves_per_s_threads": len(bw) / t_thr,
                                "solves_per_s_sequential": len(bw) / t_seq,
                                "batched": "lockstep: every inner solve of all 16 one device-driven graph launch",
                                "launch_shapes": [list(sv.tuning) for sv in bsolvers],
                                "dof_iters_per_s_batched": sum(3.0 * (sb["n_fe"] + sb["n_x"]) * sum(sb["iters"])
                                                               for sb in bst) / t_bat}
            for sv in bsolvers:
                sv.close()
            # the paper's contrast study (Sec. 4.2): Hashin's neutral inclusion at N = 128, tol 1e-7,
            # K_i / K_c from 1e-5 to 1e5 (coating modulus from the neutrality condition), linear CG
            # with the paper's identity and the 3x3-block enriched preconditioner; the paper prints
            # 1316 (K_i/K_c = 1e-5) and 16081 (1e5) X-FEM iterations
            sweep = []
            eh1 = np.array([[1.0, 1.0, 1.0, 0.0, 0.0, 0.0]])
            for ratio in (1e-5, 1e-3, 1e-1, 10.0, 1e3, 1e5):
                Lr, phr, ellr = synth.hashin_contrast(128, ratio)
                row = {"K_i/K_c": ratio}
                for enr in ("identity", "block3"):
                    sv = Solver((128, 128, 128), ellr, precision="fp32", tol=1e-7, maxit=100000,
                                enr_precond=enr)
                    sv.set_microstructure_phases(Lr, phr)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    o1 = sv.solve(eh1, u=False)
                    torch.cuda.synchronize()
                    row["iters_" + enr] = int(o1["stats"]["iters"][0])
                    row["ms_" + enr] = 1e3 * (time.perf_counter() - t0)
                    row["converged_" + enr] = bool(o1["converged"])
                    if enr == "identity":
                        row["K_eff_minus_1"] = float(o1["mean_stress"][0, :3].sum() / 9.0 - 1.0)
                    sv.close()
                sweep.append(row)
            extra["hashin_contrast_sweep"] = sweep
            # Hashin's neutral inclusion (three phases, two interfaces) at N = 128, tol 1e-7,
            # eps_bar = I: K_eff against K_matrix = 1 and the iteration counts of the three schemes
            # (the paper prints 48 for linear CG, 60 for nonlinear CG, 115 for Barzilai-Borwein and
            # 668 for the basic scheme)
            Lh, phh, ellh = synth.hashin_neutral_inclusion(128)
            eh = np.array([[1.0, 1.0, 1.0, 0.0, 0.0, 0.0]])
            hashin = {"N": 128, "tol": 1e-7}
            runs = [("fp64", "cg", {}), ("fp64", "nlcg", {}), ("fp64", "bb", {}), ("fp64", "basic", {}),
                    ("fp32", "cg", {})]
            # every Barzilai-Borwein step rule (the paper prints no formula; 115 iterations)
            runs += [("fp64", "bb", {"bb_rule": r}) for r in ("bb2", "alt", "bb1e", "bb2e")]
            runs += [("fp64", "bb", {"bb_cycle": m}) for m in (2, 3, 4)]
            for prec, scheme, kw in runs:
                sv = Solver((128, 128, 128), ellh, precision=prec, tol=1e-7, scheme=scheme, maxit=5000, **kw)
                sv.set_microstructure_phases(Lh, phh)
                sv.solve(eh, u=False)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                oh = sv.solve(eh, u=False)
                torch.cuda.synchronize()
                key = prec + "_" + scheme + "".join("_%s%s" % (k.replace("bb_", ""), v) for k, v in kw.items())
                hashin[key] = {"iters": int(oh["stats"]["iters"][0]), "converged": bool(oh["converged"]),
                               "K_eff_minus_K_matrix": float(oh["mean_stress"][0, :3].sum() / 9.0 - 1.0),
                               "ms": 1e3 * (time.perf_counter() - t0)}
                hashin["enriched_node_share"] = sv.num_enriched / 128 ** 3
                sv.close()
            extra["hashin_neutral_inclusion"] = hashin
            # precision at scale (config 5): the 256^3 fibres and the 384^3 tilted laminate, one
            # FP32-refined six-case solve each (set-up excluded), and their preconditioner's device
            # time per right-hand side and HBM fraction from a traced repeat
            scale5 = {}
            for name in ("fibers60", "laminate"):
                w5 = synth.make_workload(name)
                n5 = tuple(w5["n"])
                N5 = int(np.prod(n5))
                sv = Solver(n5, precision="fp32", tol=1e-8)
                sv.set_microstructure(w5["L"], w5["lame_minus"], w5["lame_plus"])
                sv.effective_stiffness()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                C5, st5 = sv.effective_stiffness()
                torch.cuda.synchronize()
                t5 = time.perf_counter() - t0
                sv.profile(True)
                sv.effective_stiffness()
                p5 = sv.profile_read()
                sv.profile(False)
                pm, _, pu = p5["prec_f32"]
                nX5 = sv.num_enriched
                bps = 48.0 * (N5 + nX5) * pu / (pm / 1e3) if pm > 0 else 0.0
                scale5[name] = {"grid": list(n5), "n_enriched": nX5, "solves_per_s": 1.0 / t5,
                                "cg_iters": int(sum(st5["iters"])), "converged": bool(st5["converged"]),
                                "prec_ms_per_rhs": pm / max(pu, 1),
                                "prec_frac_of_measured_hbm": bps / 1e9 / load_peaks()[0],
                                "prec_path": "five-pass (the fused y-z plane passes cover square planes of 32 ... 128 nodes)"}
                sv.close()
                del w5
            extra["precision_at_scale"] = scale5
            # the paper's caching trade-off: cut-tet element matrices cached (option cut_cache)
            # against their action recomputed from the per-side moments at every apply (default)
            cc = {"cache_bytes": 1200 * info["ncut"]}
            for cached in (True, False):
                sv = Solver(n, precision="fp32", tol=args.tol, cut_cache=cached)
                sv.set_microstructure(L_d, lm, lp, s_d)
                sv.effective_stiffness()
                sv.profile(True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                Cc, _ = sv.effective_stiffness()
                torch.cuda.synchronize()
                tc = time.perf_counter() - t0
                pc = sv.profile_read()
                sv.profile(False)
                key = "cached" if cached else "on_the_fly"
                cc["solves_per_s_" + key] = 1.0 / tc
                cc["cut_ms_per_launch_" + key] = pc["apply_cut_f32"][0] / max(pc["apply_cut_f32"][1], 1)
                cc["ceff_" + key] = Cc
                sv.close()
            cc["ceff_rel_diff"] = float(np.abs(cc.pop("ceff_cached") - cc["ceff_on_the_fly"]).max()
                                        / np.abs(cc["ceff_on_the_fly"]).max())
            cc.pop("ceff_on_the_fly")
            extra["cut_cache"] = cc
            # cuFFT (torch.fft) R2C + C2R of the same 3 x 6 FP32 fields, beside the preconditioner
            x = torch.randn(18, *n, device=dev, dtype=torch.float32)
            for _ in range(3):
                torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=n, dim=(1, 2, 3))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=n, dim=(1, 2, 3))
            e1.record()
            torch.cuda.synchronize()
            pms, _, punits = prof["prec_f32"]
            extra["fft_baseline"] = {"cufft_r2c_c2r_ms_per_rhs": e0.elapsed_time(e1) / 10 / 6,
                                     "xfft_precondition_ms_per_rhs": pms / max(punits, 1),
                                     "note": "cuFFT: 3 fields R2C + C2R per RHS (no Green solve); xfft: "
                                             "the whole preconditioner (3 passes, Green solve, fused "
                                             "update and dot product)"}
            del x
        cpu = None
        if not args.no_cpu and world == 1:
            try:
                cpu = cpu_baseline(args.cpu_n, args.tol, dev)
            except Exception as exc:  # report, never fail the GPU line
                cpu = {"error": repr(exc)}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": list(n), "n_rhs": 6,
                           "precision": "FP32 PCG; residuals of the FP64 iterate in double-word arithmetic; "
                                         "FP64 CG scalars",
                           "enriched_preconditioner": {"block3": "3x3 node blocks of the enriched reference "
                                                                 "Gram matrix, inverted in FP64",
                                                       "identity": "the paper's identity on the scaled "
                                                                   "DOFs"}[args.enr],
                           "tol": args.tol, "n_enriched": nX, "n_cut_tets": info["ncut"],
                           "launch_shapes": dict(zip(("cut_blocks", "cut_rhs_per_launch", "prec_rhs_per_group"),
                                                     solver.tuning)),
                           "l2": "inputs larger than L2 (about 1.3 GB of fields per step)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "dof_iters_per_s": dofit_rate, "cg_iters_per_step": steps_iters / args.steps,
                "refine_steps": info.get("refine"),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                "clocks": clocks}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
