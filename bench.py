#!/usr/bin/env python
"""Benchmark of the multilevel BDDC hot path: time to a 1e-8 relative residual.

One step = the whole path on one synthetic problem: set-up (index analysis, element
matrices, sub-assembly, batched factorisation, coarse basis, coarse matrix, coarsest
factorisation) followed by the PCG solve to ||r|| / ||g|| <= 1e-8 and interior recovery.
Workload: 3D linear elasticity, 48^3 trilinear hexes (345,744 free DOFs), clamped at x = 0,
gravity load, per-element E = 10^(3U) (seed 2), nu = 0.3, 4^3 cubic subdomains of 12^3,
corner + edge + face-average constraints, two-level BDDC.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

The default arm reports the mixed-precision form (FP32 factors and preconditioner, FP64
Krylov, FP64 Schur operator via refinement, FP64 coarsest level) as `value`, and the plain
FP64 form beside it.  `--impl reference` times the CPU oracle on a bounded sample.
Under torchrun every rank solves its own replica (the path is not sharded across GPUs).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF/s and time-to-1e-8 rel residual, mixed-prec batched vs plain FP64, 1×GB300"
UNIT = "DOF/s"
WORKLOADS = {
    "elasticity3d_48": "3D elasticity, 48^3 Q1 hexes, 345,744 free DOFs, 64 cubic subdomains of 12^3, "
                       "corners+edges+faces, two-level BDDC, PCG to 1e-8",
    "elasticity3d_24": "3D elasticity, 24^3 Q1 hexes, 8 cubic subdomains of 12^3 (profiling case), "
                       "corners+edges+faces, two-level BDDC, PCG to 1e-8",
    "stokes_cavity_32": "3D lid-driven cavity Stokes, 32^3 Taylor-Hood Q2-Q1 hexes, 786,077 free DOFs, "
                        "512 cubic subdomains of 4^3, corners+edges+faces, two-level BDDC, "
                        "FGMRES (mixed) / BiCGstab (FP64) to 1e-8",
    "stokes_cavity_32_3lev": "3D lid-driven cavity Stokes, 32^3 Q2-Q1, 512/64/1 subdomains, three-level BDDC, "
                             "FGMRES (mixed) / BiCGstab (FP64) to 1e-8",
    "stokes_cavity_32_4lev": "3D lid-driven cavity Stokes, 32^3 Q2-Q1, 512/64/8/1 subdomains, four-level BDDC, "
                             "FGMRES (mixed) / BiCGstab (FP64) to 1e-8",
}
WORKLOAD = "elasticity3d_48"
TOL = 1e-8
# One complete oracle set-up + solve of the 48^3 workload (oracle.bddc.Bddc, tol 1e-8, 51 PCG
# iterations), timed once, against the sample estimate on the same machine: the estimate is
# pessimistic by the stated ratio.
ORACLE_VALIDATION = {"full_solve_s": 254.7, "setup_s": 93.1, "solve_s": 161.6, "cores": 8,
                     "machine": "x86-64 build container, 8 cores", "sample_estimate_s": [362.5, 397.0],
                     "estimate_over_measured": [1.42, 1.56]}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (the slowest replica's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(n_free: int, world: int, ms: float) -> float:
    """Whole-job DOF/s: every rank solves its own replica of n_free DOFs in ms (max over ranks)."""
    return n_free * world / (ms * 1e-3)


def workload_config(prob, extra=None):
    cfg = {
        "workload": WORKLOADS[WORKLOAD],
        "n_free": int(prob.n_free),
        "n_subdomains": int(prob.n_parts[0]),
        "levels": int(prob.n_levels),
        "tol": TOL,
        "l2": "inputs larger than L2 (factors >= 6.7 GB) and a 256 MB L2 flush between steps",
        "mesh_inputs": "host arrays (the index analysis of the set-up runs on the host); rhs resident on device",
    }
    if extra:
        cfg.update(extra)
    return cfg


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return (float(pk["hbm_gbs"]), float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1692.8))),
                "measured")
    except Exception:
        return 6800.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def traffic_ratio(cls):
    """DRAM bytes per algorithmic unit of the roofline kernel class from the committed ncu summary:
    per algorithmic byte for the sweeps (profiles/trsv_sweep_traffic.json) and the factor products
    (profiles/trmv_schur_traffic.json), per FP32-equivalent flop for the tensor-core update
    (profiles/update_tc2_traffic.json); None when the kernel source changed since the counters
    were taken."""
    from paper_1201_5991_gb300 import capi
    if cls == capi.PROF_TRSV:
        fname, src_name, key = "trsv_sweep_traffic.json", "sweep.cu", "traffic_over_algorithmic"
    elif cls == capi.PROF_TRSV_IFACE:
        fname, src_name, key = "trsv_sweep_traffic.json", "sweep.cu", "traffic_over_algorithmic_interface"
    elif cls == capi.PROF_TC_UPDATE:
        fname, src_name, key = "update_tc2_traffic.json", "update_tc.cu", "traffic_over_fp32_flop"
    else:
        fname, src_name, key = "trmv_schur_traffic.json", "trmv.cu", "traffic_over_algorithmic"
    path = os.path.join(ROOT, "profiles", fname)
    try:
        with open(path) as fh:
            rec = json.load(fh)
        src = open(os.path.join(ROOT, "paper_1201_5991_gb300", "csrc", src_name), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec.get("source_sha256", rec.get("sweep_cu_sha256")):
            return None
        return float(rec.get(key, rec.get("traffic_over_algorithmic")))
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(prob, iterations: int, n_sample: int = 4, sample_iters: int = 3):
    """Time the FP64 oracle on a bounded sample and extrapolate to the whole solve.

    Sample: the oracle's full index analysis; sub-assembly and set-up (Cholesky of K_II,
    LU of the saddle-point matrix, coarse basis) of n_sample subdomains spread over the mesh;
    sample_iters Krylov iterations' subdomain solves (Schur apply + preconditioner) for the same
    subdomains, after one untimed warm-up solve (BLAS threads, first-touch pages).
    Estimate = analysis + n_sub * mean setup + iterations * n_sub * mean iteration.
    Returns (estimate_s, description, elapsed_s).
    """
    import numpy as np
    import scipy.linalg as sla

    from oracle import fem
    from oracle import maps as om
    from oracle.bddc import _local_matrices

    t0 = time.perf_counter()
    mesh = om.mesh_level1(prob)
    mp = om.analyze(mesh, prob.constraints)
    t_analysis = time.perf_counter() - t0
    Ke = fem.element_matrices(prob)
    ns = prob.n_parts[0]
    sample = sorted(set(int(round(x)) for x in np.linspace(0, ns - 1, min(n_sample, ns))))
    sub_maps = om.LevelMaps(**{**mp.__dict__})
    sub_maps.sub_dofs = [mp.sub_dofs[s] for s in sample]
    sub_maps.sub_elems = [mp.sub_elems[s] for s in sample]
    mesh_s = om.LevelMesh(**{**mesh.__dict__, "n_sub": len(sample)})
    t1 = time.perf_counter()
    K = _local_matrices(mesh_s, sub_maps, Ke)
    facts = []
    for k, s in enumerate(sample):
        nI = mp.sub_nI[s]
        Ks = K[k]
        C = mp.sub_C[s]
        n, nc = Ks.shape[0], C.shape[0]
        kii = sla.lu_factor(Ks[:nI, :nI])   # the oracle's own routine for K_II (dense LU)
        Sd = np.zeros((n + nc, n + nc))
        Sd[:n, :n] = Ks
        Sd[:n, n:] = C.T
        Sd[n:, :n] = C
        lu = sla.lu_factor(Sd)
        rhs = np.zeros((n + nc, nc))
        rhs[n:] = np.eye(nc)
        sla.lu_solve(lu, rhs)
        facts.append((kii, lu, Ks, nI, n, nc))
    t_setup = (time.perf_counter() - t1) / len(sample)

    def one_iteration(kii, lu, Ks, nI, n, nc):
        x = np.ones(n - nI)
        w = sla.lu_solve(kii, Ks[:nI, nI:] @ x)
        _ = Ks[nI:, nI:] @ x - Ks[nI:, :nI] @ w
        r = np.zeros(n + nc)
        r[nI:n] = 1.0
        sla.lu_solve(lu, r)

    one_iteration(*facts[0])   # warm-up
    t2 = time.perf_counter()
    for _ in range(sample_iters):
        for f in facts:
            one_iteration(*f)
    t_iter = (time.perf_counter() - t2) / (len(sample) * sample_iters)
    per_it = 2 if prob.physics == 2 else 1   # BiCGstab: two operator and preconditioner applications
    est = t_analysis + ns * t_setup + per_it * iterations * ns * t_iter
    elapsed = time.perf_counter() - t0
    desc = (f"index analysis of all {ns} subdomains + set-up of {len(sample)} of {ns} subdomains + "
            f"{sample_iters} iterations' subdomain solves for the same {len(sample)}, extrapolated to {ns} "
            f"subdomains x {iterations} Krylov iterations x {per_it} applications ({elapsed:.1f} s of CPU work)")
    return est, desc, elapsed


def cpu_cores():
    return os.cpu_count() or 1


# ----------------------------------------------------------------------------- GPU arm
def multi_rhs_leg(stream, dev, reps: int = 2):
    """64^3 elasticity with 16 seeded load cases (512 subdomains of 8^3), mixed precision, tol 1e-8:
    set-up plus the 16-column solve, and the solve of one column alone, timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1201_5991_gb300 import meshgen
    from paper_1201_5991_gb300.solver import BddcSolver

    p5 = meshgen.config("elasticity3d_64_16rhs")
    F = torch.tensor(np.ascontiguousarray(p5.f.T), dtype=torch.float64, device=dev)
    F1 = F[0].contiguous()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    s = BddcSolver(p5, precision="mixed", stream=stream)   # warm-up: graphs, block buffers, tuning cache
    s.solve(F, tol=TOL)
    s.solve(F1, tol=TOL)
    def setup_and_solve():
        q = BddcSolver(p5, precision="mixed", stream=stream)
        q.solve(F, tol=TOL)
        return q

    step, one, many = [], [], []
    for _ in range(reps):
        ms, s2 = timed(setup_and_solve)
        step.append(ms)
        st16 = s2.last_stats
        del s2
        one.append(timed(lambda: s.solve(F1, tol=TOL))[0])
        st1 = s.last_stats
        many.append(timed(lambda: s.solve(F, tol=TOL))[0])
    t_step, t1, t16 = min(step), min(one), min(many)
    return {
        "workload": "3D elasticity, 64^3 Q1 hexes, 811,200 free DOFs, 512 cubic subdomains of 8^3, "
                    "corners+edges+faces, two-level BDDC, 16 seeded load cases, PCG to 1e-8",
        "ms_setup_plus_16_rhs": t_step, "ms_solve_16_rhs": t16, "ms_solve_1_rhs": t1,
        "dof_rhs_per_s": p5.n_free * 16 / (t_step * 1e-3),
        "solve_16_over_1": t16 / t1, "iterations_16": st16.iterations, "iterations_1": st1.iterations,
        "block": "8 columns per pass over the factors",
    }



def stokes_leg(stream, dev, reps: int = 2):
    """The Stokes lid-driven cavity (32^3 Taylor-Hood Q2-Q1 hexes, 786,077 free DOFs, 512 cubic
    subdomains), mixed precision, flexible GMRES to 1e-8, with two, three and four levels
    (512 / 1, 512 / 64 / 1, 512 / 64 / 8 / 1 subdomains): set-up plus solve of one right-hand side,
    timed with CUDA events, best of reps after a warm-up (graphs, tuning cache)."""
    import numpy as np
    import torch

    from paper_1201_5991_gb300 import meshgen
    from paper_1201_5991_gb300.solver import BddcSolver

    out = {"workload": "3D Stokes lid-driven cavity, 32^3 Q2-Q1 hexes, 786,077 free DOFs, 512 cubic subdomains "
                       "of 4^3, signed Cholesky local saddle points, flexible GMRES to 1e-8"}
    for name, key in (("stokes_cavity_32", "levels_2"), ("stokes_cavity_32_3lev", "levels_3"),
                      ("stokes_cavity_32_4lev", "levels_4")):
        p = meshgen.config(name)
        F = torch.tensor(np.ascontiguousarray(p.f[:, 0]), dtype=torch.float64, device=dev)

        def step():
            s = BddcSolver(p, precision="mixed", stream=stream)
            s.solve(F, tol=TOL)
            return s

        warm = step()   # graphs, block buffers, tuning cache of these level shapes
        del warm
        best, st = None, None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s = step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if best is None or ms < best:
                best, st = ms, s.last_stats
            del s
        out[key] = {"ms": round(best, 2), "dof_per_s": p.n_free / (best * 1e-3), "iterations": st.iterations,
                    "setup_ms": round(st.analysis_ms + st.prepare_ms + st.factor_ms, 2),
                    "solve_ms": round(st.solve_ms, 2), "rel_residual": st.rel_residual}
    return out


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1201_5991_gb300 import capi, meshgen
    from paper_1201_5991_gb300.solver import BddcSolver

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = meshgen.config(WORKLOAD)
    f = torch.tensor(prob.f[:, 0], dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    L = capi.lib()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def one_step(precision, profile=0):
        s = BddcSolver(prob, precision=precision, stream=stream, profile=profile)
        u = s.solve(f, tol=TOL)
        return s, u

    def timed(precision, steps, warmup, profile=0, clocks=False):
        for _ in range(warmup):
            s, u = one_step(precision)
            del s, u
        torch.cuda.synchronize()
        barrier()
        sampler = ClockSampler(local_rank) if clocks else None
        if sampler:
            sampler.start()
        times, stats = [], []
        launches0 = L.bddc_kernel_launches()
        prof = [0.0, 0, 0.0]
        cls = {c: [0.0, 0, 0.0, 0.0] for c in range(capi.PROF_CLASSES)}
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s, u = one_step(precision, profile)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            st = s.stats()
            stats.append(st)
            for c, acc in cls.items():
                acc[0] += st.prof_ms[c]
                acc[1] += st.prof_launches[c]
                acc[2] += st.prof_bytes[c]
                acc[3] += st.prof_flops[c]
            del s, u
        launches = (L.bddc_kernel_launches() - launches0) / max(steps, 1)
        # the roofline kernel: the single kernel class with the largest share of the step
        dom = max((capi.PROF_TRSV, capi.PROF_TRSV_IFACE, capi.PROF_TRMV, capi.PROF_TC_UPDATE),
                  key=lambda c: cls[c][0])
        prof = [cls[dom][0], cls[dom][1], cls[dom][2], dom, cls]
        torch.cuda.synchronize()
        barrier()
        clk = sampler.stop() if sampler else None
        ms = max_over_ranks(sum(times) / len(times), world, dev)
        last_times[:] = [round(t, 2) for t in times]
        return ms, stats, launches, prof, clk

    last_times = []
    ms, stats, launches, prof, clk = timed("mixed", args.steps, args.warmup, profile=1, clocks=True)
    step_ms = list(last_times)
    value = weak_scaling_value(prob.n_free, world, ms)
    st0 = stats[-1]

    # plain FP64 form, same workload (fewer steps: its set-up is FP64-ALU bound)
    pk = max(1, min(args.steps, args.plain_steps))
    if args.no_plain:
        ms64, st64 = None, None
    else:
        ms64, stats64, _, _, _ = timed("fp64", pk, 1)
        st64 = stats64[-1]

    # accuracy of the timed mixed form against the plain FP64 form on the same problem (both to
    # 1e-8; outside the timed region)
    err = None
    if st64 is not None:
        s_m, u_m = one_step("mixed")
        s_p, u_p = one_step("fp64")
        err = {"rel_l2_error_mixed_vs_plain_fp64": float(torch.linalg.norm(u_m - u_p) / torch.linalg.norm(u_p)),
               "note": "both solved to ||g - S u|| / ||g|| <= 1e-8; parity with the FP64 oracle at 1e-12 is in tests/"}
        del s_m, u_m, s_p, u_p

    # batching ablation (outside the timed region): level-1 sweeps and CUDA-core factorisation
    # in one launch for all subdomains vs one launch per subdomain
    ablation = None
    if not args.no_ablation:
        try:
            s_ab = BddcSolver(prob, precision="mixed", stream=stream)
            ablation = {k: round(v, 3) for k, v in s_ab.batching_ablation().items()}
            del s_ab
        except capi.BddcError as e:
            ablation = {"unavailable": str(e)}

    # the 16-load-case workload (64^3 elasticity, 512 subdomains): the right-hand sides solved as
    # blocks of 8 columns (every factor tile read once per block and iteration) against one column
    multi = None
    if not args.no_multi_rhs:
        multi = multi_rhs_leg(stream, dev)

    # the Stokes cavity (indefinite local problems) with two, three and four levels
    stokes = None
    if not args.no_stokes:
        try:
            stokes = stokes_leg(stream, dev)
        except Exception as e:   # reported, never fatal for the headline line
            stokes = {"unavailable": f"{type(e).__name__}: {e}"}

    # end to end through the public host-buffer entry point
    fh = np.ascontiguousarray(prob.f[:, 0])
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = BddcSolver(prob, precision="mixed", stream=stream)
        u = s.solve_host(fh, tol=TOL)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        del s
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), world, dev)
    mesh_bytes = prob.coords.nbytes + prob.conn.nbytes + prob.coef.nbytes + prob.dirichlet.nbytes

    hbm, tc_peak, peak_kind = load_peaks()
    dom, cls = prof[3], prof[4]
    tensor = dom == capi.PROF_TC_UPDATE
    ratio = traffic_ratio(dom)
    if tensor:   # three FP16 tensor-core products per FP32-equivalent multiply-add (scaled hi/lo split)
        achieved = 3.0 * cls[dom][3] / (prof[0] * 1e-3) / 1e12 if prof[0] > 0 else 0.0
        units = cls[dom][3]   # FP32-equivalent flops: the DRAM bytes are the output tiles, read and written once
    else:
        achieved = prof[2] / (prof[0] * 1e-3) / 1e9 if prof[0] > 0 else 0.0
        units = prof[2]
    traffic = ratio * units / max(prof[1], 1) if ratio is not None else None
    names = {capi.PROF_TRSV: "k_sweep<float> forward/backward over interior block rows (Schur operator; "
                             "streaming triangular sweeps, TMA-staged tiles)",
             capi.PROF_TRSV_IFACE: "k_sweep<float> forward/backward over interface block rows (subdomain corrections)",
             capi.PROF_COARSE: "coarsest-level solves (k_coarse_apply with the explicit FP32 inverse of the "
                               "FP64 coarse factor, else sweeps over it)",
             capi.PROF_TRMV: "inner Schur operator: k_schur_symv_rows + _cols over the explicit augmented Schur "
                             "complement, else k_trmv_t + k_trmv_n with the stored interface factor",
             capi.PROF_SPMV: "k_spmv (FP64 CSR products with K_i)",
             capi.PROF_FACTOR: "factorisation steps on CUDA cores (diagonal blocks: k_potrf_diag, k_trsm_panel, "
                               "k_syrk_update; k_block_inverse, k_split_inverse, k_split_panel)",
             capi.PROF_TC_PANEL: "k_update_tc2 as the panel solve A(i, D) X^T S_D below each 256 x 256 diagonal "
                                 "block (FP32-equivalent flops of the triangular solves it replaces)",
             capi.PROF_TC_UPDATE: "k_update_tc2 (rank-256 and rank-512 trailing updates of 512-wide super-panels "
                                  "on tcgen05, scaled two-part FP16 products, persistent, TMEM double-buffered)"}
    kernel_classes = {}
    for c, (cms, cl, cb, cf) in cls.items():
        if cl == 0:
            continue
        e = {"kernel": names[c], "ms_per_step": round(cms / args.steps, 3), "launches_per_step": cl / args.steps,
             "share_of_step": round(cms / args.steps / ms, 4) if ms > 0 else None}
        if cb > 0:
            e["achieved_GBps"] = round(cb / (cms * 1e-3) / 1e9, 1)
            e["frac_of_hbm"] = round(cb / (cms * 1e-3) / 1e9 / hbm, 4)
        if cf > 0:
            e["achieved_TFLOPs_fp32"] = round(cf / (cms * 1e-3) / 1e12, 2)
        if c in (capi.PROF_TC_UPDATE, capi.PROF_TC_PANEL) and cf > 0:
            e["achieved_TFLOPs_fp16_mma"] = round(3.0 * cf / (cms * 1e-3) / 1e12, 1)
            e["frac_of_tensor_peak"] = round(3.0 * cf / (cms * 1e-3) / 1e12 / tc_peak, 4)
        kernel_classes[{capi.PROF_TRSV: "trsv_interior", capi.PROF_TRSV_IFACE: "trsv_interface",
                        capi.PROF_COARSE: "trsv_coarsest", capi.PROF_TRMV: "trmv", capi.PROF_SPMV: "spmv",
                        capi.PROF_FACTOR: "factor_cuda_cores", capi.PROF_TC_UPDATE: "tc_update",
                        capi.PROF_TC_PANEL: "tc_panel_solve"}[c]] = e
    peak = tc_peak if tensor else hbm
    roofline = {
        "kernel": names[dom],
        "bound": "tensor" if tensor else "hbm",
        "achieved": round(achieved, 1),
        "peak": peak,
        "peak_kind": (peak_kind + (" bf16 sustained (fp16 dense rate = bf16)" if tensor else " copy bandwidth")),
        "unit": "TFLOP/s" if tensor else "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": traffic,
        "launches_per_step": prof[1] / max(args.steps, 1),
        "algorithmic_bytes_per_launch": None if tensor else prof[2] / max(prof[1], 1),
        "algorithmic_fp32_flops_per_launch": cls[dom][3] / max(prof[1], 1) if tensor else None,
        "avg_launch_ms": prof[0] / max(prof[1], 1),
        "share_of_step": round(prof[0] / args.steps / ms, 4) if ms > 0 else None,
        "classes": kernel_classes,
    }

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        est, desc, elapsed = oracle_sample(prob, st64.iterations if st64 else st0.iterations)
        cpu = {"value": prob.n_free / est, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": desc,
               "sample_elapsed_s": elapsed, "est_time_to_solution_s": est, "validation": ORACLE_VALIDATION}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed-f32/f64",
        "data": "synthetic",
        "config": workload_config(prob, {"precision": "mixed (FP32 factors, FP64 Krylov and Schur operator)",
                                         "replicas": world}),
        "time_to_1e-8_ms": ms,
        "step_ms": step_ms,
        "iterations": st0.iterations,
        "rel_residual": st0.rel_residual,
        "setup_ms": st0.analysis_ms + st0.prepare_ms + st0.factor_ms,
        "analysis_ms": st0.analysis_ms,
        "prepare_ms": st0.prepare_ms,
        "factor_ms": st0.factor_ms,
        "solve_ms": st0.solve_ms,
        "refine_steps": st0.refine_steps,
        "inner_steps": st0.inner_steps,
        "autotuned_sweeps": {f"level{l + 1}_{'interior' if part == 0 else 'interface'}":
                             {"ctas_per_sm": st0.sweep_ctas[2 * l + part], "deep_ring": st0.sweep_deep[2 * l + part],
                              "longest_first": st0.sweep_order[2 * l + part]}
                             for l in range(st0.n_levels) for part in range(2)},
        "outer_iterations": st0.outer_iterations,
        "kappa_estimate": (st0.lambda_max / st0.lambda_min if st0.lambda_min > 0 and prob.physics != 2
                           else None),
        "plain_fp64": None if st64 is None else {
            "value": prob.n_free * world / (ms64 * 1e-3), "ms_per_step": ms64, "steps": pk,
            "iterations": st64.iterations, "setup_ms": st64.analysis_ms + st64.prepare_ms + st64.factor_ms,
            "solve_ms": st64.solve_ms, "speedup_mixed_vs_plain": ms64 / ms},
        "e2e": {"value": prob.n_free * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(prob.n_free * 8 + mesh_bytes), "d2h_bytes_per_step": int(prob.n_free * 8)},
        "gpu_launches": int(round(launches)),
        "batching_ablation": ablation,
        "multi_rhs": multi,
        "stokes_cavity": stokes,
        "accuracy": err,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1201_5991_gb300 import meshgen
    prob = meshgen.config(WORKLOAD)
    iters = args.ref_iterations
    if args.warmup > 0:
        oracle_sample(prob, iters)          # one untimed sample warms BLAS / allocators
    ests, elapsed = [], []
    desc = ""
    for _ in range(args.steps):
        est, desc, el = oracle_sample(prob, iters)
        ests.append(est)
        elapsed.append(el)
    est = sum(ests) / len(ests)
    value = prob.n_free / est
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(elapsed) / len(elapsed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(prob, {"precision": "FP64 oracle (dense LAPACK per subdomain)"}),
        "impl": "reference",
        "note": ("each step times a bounded sample of the oracle's solve (ms_per_step is the sample's elapsed "
                 "time); value is the sample's estimate of the whole set-up plus solve, est_time_to_solution_ms"),
        "est_time_to_solution_ms": 1e3 * est,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": desc,
                         "validation": ORACLE_VALIDATION},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    global WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--ref-iterations", type=int, default=51)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 form (profiling runs)")
    ap.add_argument("--no-ablation", action="store_true", help="skip the batching ablation (profiling runs)")
    ap.add_argument("--no-multi-rhs", action="store_true", help="skip the 16-load-case leg (profiling runs)")
    ap.add_argument("--no-stokes", action="store_true", help="skip the Stokes cavity leg (profiling runs)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    args = ap.parse_args()
    WORKLOAD = args.workload
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
