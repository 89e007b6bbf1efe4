#!/usr/bin/env python
"""Benchmark: DOFs/s to l2 relative residual 1e-8 on one GB300.

Workload (one step = the whole hot path over one batch of input): the
distorted-mesh Riesz maps on an 8x8x8 hexahedral mesh of the unit cube with
10% random interior-vertex perturbation, p = 7, alpha = beta = 1, N(0,1)
right-hand sides:
  * H(grad): 185,193 lattice DOFs, SC-PAFW vertex stars with ICC(0) on the
    static-condensation pattern of the auxiliary operator + P1 coarse;
  * H(curl): 545,832 lattice DOFs, SC-PH (edge-star Cholesky + vertex-star
    ICC(0) potential patches) + P1 coarse.
One step solves both from a zero initial guess.  The headline variant is
the mixed-precision one (FP32 preconditioner inside FP64 flexible CG); the
plain FP64 solver is timed alongside ("variants").

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the CPU oracle (plain FP64 NumPy/SciPy) on a bounded
sample of the same workload (3x3x3 mesh, same p, perturbation and solvers).
"""

from __future__ import annotations

import argparse
import concurrent.futures
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOFs/s to rel. residual 1e-8: mixed/batched/learned vs plain FP64, 1 GB300"
N_CELLS, DEGREE, PERTURB = 8, 7, 0.1
WORKLOAD = "Riesz maps H(grad)+H(curl), 8x8x8 hex, 10% interior-vertex perturbation, p=7"
SPACES = [
    ("hgrad", 0, dict(static_condensation=1, factor=1)),
    ("hcurl", 1, dict(static_condensation=1, factor=1, decomposition=1)),
]
# fp64: the plain FP64 solver (FP64 preconditioner, FP64 operator apply, CG);
# fp64_df: the same with the double-float apply; mixed_fp32 (headline): FP32
# preconditioner inside FP64 flexible CG, double-float apply
VARIANTS = {"fp64": dict(precision=0, flexible=0, arith=0),
            "fp64_df": dict(precision=0, flexible=0, arith=1),
            "mixed_fp32": dict(precision=1, flexible=1, arith=1)}
DTYPES = {"fp64": "f64 (CG, apply, preconditioner)",
          "fp64_df": "f64 CG and preconditioner, double-float (2 x f32) apply",
          "mixed_fp32": "f64 CG, double-float (2 x f32) apply, f32 preconditioner"}
HEADLINE = "mixed_fp32"
# dram__bytes_read.sum + dram__bytes_write.sum of one H(grad) general apply
# (apply_kernel<0,7> and its assembly, double-float, 8^3 cells) in an ncu
# capture of this workload (profiles/apply_kernel_hgrad_8cubed_p7.md)
APPLY_TRAFFIC_BYTES = 53_107_712
FP64_PEAK_TFLOPS = 1.20   # measured FP64 FMA throughput of a GB300 (DFMA throughput probe)
# Algorithmic HBM bytes per lattice DOF per CG iteration of the whole solve:
# CG vectors ~80 B (FP64, fused updates and dots), operator apply 16 B (x in,
# y out), condensation ~4 vector passes, patch factors nnz(L)/DOF x value
# bytes (~19 nnz per DOF for H(grad) SC vertex stars at p = 7) + 2 vector
# passes, coarse ~0: ~260 B with an FP64 preconditioner, ~185 B with FP32.
SOLVE_BYTES_PER_DOF_ITER = {"fp64": 260.0, "fp64_df": 260.0, "mixed_fp32": 185.0}


def measured_peaks():
    """HBM copy bandwidth and BF16 GEMM rate measured on the GB300s
    (MEASURED_PEAKS.json beside this file), else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}
# The general apply computes in double-float (pairs of FP32, ~48 bits) on the
# FP32 pipe.  Its ceiling from unit counts and clocks: 152 SMs x 128 FP32
# lanes x 2.07 GHz = 40.3 T FP32 instructions/s; a double-float FMA (2 FP64-
# equivalent flops) takes 15 FP32 instructions -> 5.37 TFLOP/s FP64-equivalent.
DF_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 15 * 2 / 1e12


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's time: N independent replicas finish with it."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, dofs: int, ms: float) -> float:
    """Whole-job DOFs/s: every rank solves its own steps x dofs (weak
    scaling) within the slowest rank's time ms."""
    return world * steps * dofs / (ms / 1e3)


# ---------------------------------------------------------------------------
def apply_flops(k: int, p: int) -> float:
    """Algorithmic flops (FP64-equivalent) of one sum-factorised apply on one cell:
    interpolation to and from the q^3 GLL points for V^k and V^{k+1}
    (three 1D contractions each way), D-hat and D-hat^T, and the pointwise
    metric products.  The pullback metric itself is computed once at setup
    (metric_kernel) and read per apply: 8 B x (7 or 12) per point."""
    q = (3 * (p + 1) + 1) // 2
    types = {0: ["sss"], 1: ["rss", "srs", "ssr"], 2: ["srr", "rsr", "rrs"], 3: ["rrr"]}
    fma = 0
    for kk in (k, k + 1):
        for t in types[kk]:
            l = [p + 1 if c == "s" else p for c in t]
            fwd = q * l[0] * l[1] * l[2] + q * q * l[1] * l[2] + q ** 3 * l[2]
            fma += 2 * fwd
        vec = len(types[kk]) == 3
        fma += q ** 3 * (9 if vec else 1)
    nterms = {0: 3, 1: 6, 2: 3}[k]
    fma += 2 * nterms * p * (p + 1) * (p + 1) * (p + 1)   # D-hat and its transpose
    return 2.0 * fma


def cart_apply_flops(k: int, p: int) -> float:
    """Algorithmic flops (FP64-equivalent) of the Cartesian apply on one cell:
    per signed D-hat term the D-hat product (three nonzeros per row of D-hat
    in the FDM basis, two in its first row) and the D-hat^T product (one
    multiply-add per interior row, the 2P-entry line sums for the interface
    rows), plus the beta and alpha coefficient scalings.  The 2x2 B-hat
    interface blocks are not counted (a lower bound)."""
    types = {0: ["sss"], 1: ["rss", "srs", "ssr"], 2: ["srr", "rsr", "rrs"], 3: ["rrr"]}

    def size(kk):
        t = types[kk][0]
        return math.prod(p + 1 if c == "s" else p for c in t)
    s0, s1 = size(k), size(k + 1)
    nterms = {0: 3, 1: 6, 2: 3}[k]
    per_term = (3 * p - 1) * (s1 // p) + (3 * p - 1) * (s0 // (p + 1))
    macs = nterms * per_term + len(types[k]) * s0 + len(types[k + 1]) * s1
    return 2.0 * macs


def run_apply_kernels(steps, stream):
    """The operator apply alone on the axis-aligned-cell workloads (the
    Cartesian kernel pair): 32^3 H(grad) at p = 6 and 16^3 H(div) at p = 10,
    double-float and FP64.  Inputs, output and the unassembled scratch
    (> 200 MB) exceed L2, so no flush is needed between applies."""
    import torch
    from paper_2211_14284_gb300.rm import Solver
    peaks = measured_peaks()
    out = {}
    for name, k, n, p in (("hgrad_32cubed_p6", 0, 32, 6), ("hdiv_16cubed_p10", 2, 16, 10)):
        res = {}
        for aname, arith in (("df64", 1), ("fp64", 0)):
            s = Solver(k, n, p, relaxation=0, arith=arith, stream=stream)
            x = torch.randn(s.size, dtype=torch.float64, device="cuda")
            y = torch.zeros_like(x)
            for _ in range(3):
                s.apply(x, y)
            reps = max(10, 4 * steps)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                s.apply(x, y)
            ev1.record(stream)
            ev1.synchronize()
            ms = ev0.elapsed_time(ev1) / reps
            tflops = cart_apply_flops(k, p) * n ** 3 / (ms / 1e3) / 1e12
            res[aname] = {"ms_per_apply": ms, "dofs": s.size, "dofs_per_s": s.size / (ms / 1e3),
                          "tflops_fp64_equiv": tflops,
                          "alu_frac": tflops / (DF_PEAK_TFLOPS if arith else FP64_PEAK_TFLOPS),
                          "hbm_frac": 16.0 * s.size / (ms / 1e3) / (peaks["hbm_gbs"] * 1e9)}
            s.close()
        out[name] = res
    return out


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = float(f[2])
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    from paper_2211_14284_gb300 import inputs
    from paper_2211_14284_gb300.rm import Solver

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    n, p = N_CELLS, DEGREE
    X = inputs.vertices(n, perturb=PERTURB, seed=2)
    al = inputs.constant_coefficient(n)
    be = inputs.constant_coefficient(n)

    # the two problems of a step are independent: each solves on its own
    # stream, driven by its own host thread, so their latency-bound kernels
    # overlap on the GPU
    space_streams = {sname: torch.cuda.Stream() for sname, _, _ in SPACES}
    pool = concurrent.futures.ThreadPoolExecutor(max_workers=len(SPACES))
    solvers = {}
    t0 = time.time()
    for vname, vopt in VARIANTS.items():
        for sname, k, sopt in SPACES:
            solvers[(vname, sname)] = Solver(k, n, p, vertices=X, alpha=al, beta=be,
                                             stream=space_streams[sname], rtol=1e-8, max_it=1000,
                                             profile=1, deterministic=1 if args.deterministic else 0,
                                             **sopt, **vopt)
    setup_s = time.time() - t0
    sizes = {sname: solvers[(HEADLINE, sname)].size for sname, _, _ in SPACES}
    dofs = sum(sizes.values())
    bh = {sname: torch.tensor(inputs.normal_rhs(sizes[sname], 100 + k + 7 * rank),
                              dtype=torch.float64).pin_memory() for sname, k, _ in SPACES}
    bd = {s: bh[s].cuda() for s in bh}
    xd = {s: torch.zeros_like(bd[s]) for s in bd}
    xh = {s: torch.zeros_like(bh[s]).pin_memory() for s in bh}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def solve_space(vname, sname, e2e, start):
        st = space_streams[sname]
        st.wait_event(start)
        with torch.cuda.stream(st):
            if e2e:
                bd[sname].copy_(bh[sname], non_blocking=True)
            xd[sname].zero_()
            info = solvers[(vname, sname)].solve(bd[sname], xd[sname])
            if info["status"] != "RM_OK" or not info["rel_res_l2"] <= 1e-8:
                raise RuntimeError(f"{vname}/{sname} did not converge: {info}")
            if e2e:
                xh[sname].copy_(xd[sname], non_blocking=True)
            done = torch.cuda.Event()
            done.record(st)
        return sname, info, done

    def one_step(vname, e2e, stats):
        """Both problems from the main stream's current point; returns when
        the main stream has been made to wait for both."""
        start = torch.cuda.Event()
        start.record(stream)
        if args.sequential:
            results = [solve_space(vname, sname, e2e, start) for sname, _, _ in SPACES]
        else:
            results = [f.result() for f in [pool.submit(solve_space, vname, sname, e2e, start)
                                            for sname, _, _ in SPACES]]
        for sname, info, done in results:
            stream.wait_event(done)
            stats.append((sname, info))

    def timed(vname, e2e, steps, warmup):
        for _ in range(warmup):
            one_step(vname, e2e, [])
        barrier()
        total_ms = 0.0
        stats = []
        for _ in range(steps):
            flush.fill_(1.0)                           # evict the working set from L2
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            one_step(vname, e2e, stats)
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
        barrier()
        return max_over_ranks(total_ms, world, "cuda"), stats

    results = {}
    with ClockSampler(local) as clk:
        for vname in VARIANTS:
            ms, stats = timed(vname, False, args.steps, args.warmup)
            results[vname] = (ms, stats)
    clocks = clk.summary()
    e2e_ms, _ = timed(HEADLINE, True, args.steps, max(1, args.warmup // 2))

    peaks = measured_peaks()

    def summarise(vname):
        ms, stats = results[vname]
        it = {s: [i["iterations"] for (sn, i) in stats if sn == s] for s, _, _ in SPACES}
        dof_its = sum(sizes[sn] * i["iterations"] for (sn, i) in stats)
        byts = SOLVE_BYTES_PER_DOF_ITER[vname] * dof_its
        return {
            "value": job_value(world, args.steps, dofs, ms),
            "ms_per_step": ms / args.steps,
            "dtype": DTYPES[vname],
            "iterations": {s: int(statistics.median(v)) for s, v in it.items()},
            "iterations_natural": {s: int(statistics.median([i["iterations_natural"] for (sn, i) in stats
                                                            if sn == s])) for s, _, _ in SPACES},
            "solve_ms": {s: statistics.median([i["solve_ms"] for (sn, i) in stats if sn == s])
                         for s, _, _ in SPACES},
            "apply_ms_per_call": sum(i["apply_ms"] for (_, i) in stats) /
                                 max(1, sum(i["apply_calls"] for (_, i) in stats)),
            # whole-solve HBM roofline: algorithmic bytes (per DOF per iteration
            # x DOF-iterations) over the measured time, against the measured copy rate
            "hbm_frac_solve": byts / (ms / 1e3) / (peaks["hbm_gbs"] * 1e9),
            "hbm_bytes_per_dof_iter": SOLVE_BYTES_PER_DOF_ITER[vname],
        }

    head = summarise(HEADLINE)
    ms_h, stats_h = results[HEADLINE]
    launches = sum(i["kernel_launches"] for (_, i) in stats_h)
    # dominant kernel: the operator apply (double-float, ALU-bound); its average
    # duration over the timed region, from the solver's own CUDA events
    app_ms = sum(i["apply_ms"] for (_, i) in stats_h)
    app_calls = sum(i["apply_calls"] for (_, i) in stats_h)
    flops = 0.0
    for sname, k, _ in SPACES:
        calls = sum(i["apply_calls"] for (sn, i) in stats_h if sn == sname)
        flops += calls * apply_flops(k, DEGREE) * N_CELLS ** 3
    achieved = flops / (app_ms / 1e3) / 1e12
    roof = {"bound": "alu",
            "kernel": "apply_kernel + cart_assemble_kernel (sum-factorised operator, double-float on "
                      "the FP32 pipe, then the fixed-order assembly of the cell products)",
            "achieved": achieved, "peak": DF_PEAK_TFLOPS,
            "unit": "TFLOP/s (FP64-equivalent; peak = double-float FMA rate from unit counts)",
            "frac": achieved / DF_PEAK_TFLOPS,
            # DRAM bytes of one apply (ncu dram__bytes_read.sum + write.sum of
            # the two kernels, H(grad) instance, 512 cells): the pullback
            # metric (49.5 MB) plus the cell gathers and the products, no re-reads
            "traffic": APPLY_TRAFFIC_BYTES,
            "traffic_launch": "apply_kernel<0,7> + cart_assemble_kernel<0,7>, 8^3 cells, one apply (ncu)",
            "fp64_pipe_peak": FP64_PEAK_TFLOPS,
            "avg_launch_ms": app_ms / max(app_calls, 1),
            "time_share_of_step": app_ms / ms_h,
            "preconditioner_share_of_step": sum(i["precond_ms"] for (_, i) in stats_h) / ms_h,
            "hbm_frac_solve": head["hbm_frac_solve"],
            "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peaks["source"]}
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "DOFs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[HEADLINE],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice_dofs": dofs,
                   "lattice_dofs_per_space": sizes, "rtol": 1e-8,
                   "variant": HEADLINE, "l2": "flushed between steps (256 MiB write)",
                   "relaxation": "deterministic (fixed-order patch sums, branches in sequence)"
                                 if args.deterministic else "default (atomic patch scatters, concurrent branches)",
                   "parallelism": "independent replicas" if world > 1 else "1 GPU",
                   "spaces": "one after another" if args.sequential else "concurrent (a stream and host thread each)",
                   "iterations": head["iterations"], "setup_s": setup_s},
        "e2e": {"value": job_value(world, args.steps, dofs, e2e_ms), "unit": "DOFs/s",
                "h2d_bytes_per_step": 8 * dofs, "d2h_bytes_per_step": 8 * dofs},
        "gpu_launches": launches,
        "roofline": roof,
        "variants": {v: summarise(v) for v in VARIANTS},
        "clocks": clocks,
    }
    if not args.no_apply_kernels:
        line["apply_kernels"] = run_apply_kernels(args.steps, stream)
    if args.batch_count > 0:
        line["variants"]["batched"] = run_batched(args.batch_count, args.steps,
                                                  max(1, args.warmup // 2), stream)
    if args.learned_epochs > 0:
        line["variants"]["learned"] = run_learned(args.steps, max(1, args.warmup // 2),
                                                  args.learned_epochs, args.learned_size, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_full() if args.cpu_baseline_full else cpu_baseline(args, budget_s=30.0)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
def _oracle_sample():
    """The oracle's solvers on the 3x3x3 sample of the workload (same p,
    perturbation, coefficients, preconditioners)."""
    from oracle.auxiliary import assemble_aux
    from oracle.discretization import Problem
    from oracle.relaxation import SCPAFW, SCPH
    from paper_2211_14284_gb300 import inputs
    n = 3
    X = inputs.vertices(n, perturb=PERTURB, seed=2)
    al = inputs.constant_coefficient(n)
    be = inputs.constant_coefficient(n)
    out = []
    for sname, k, _ in SPACES:
        pr = Problem(k, n, DEGREE, X, al, be)
        A = pr.A_free()
        P = assemble_aux(pr)[pr.free][:, pr.free]
        M = SCPAFW(pr, P, factor="icc") if k == 0 else SCPH(pr, P)
        b = inputs.normal_rhs(pr.lat.size, 100 + k)[pr.free]
        out.append((sname, pr.lat.size, A, M, b))
    return out


def cpu_baseline(args, budget_s=30.0):
    cores = len(os.sched_getaffinity(0))
    if args.cpu_baseline_full:
        # the whole workload (one solve per space, set-up excluded), minutes
        full = cpu_baseline_full()
        v = full["value"]
        dofs = full["runs"]["all_cores"]["dofs"]
        print(json.dumps({
            "metric": METRIC, "value": v, "unit": "DOFs/s", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * dofs / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice_dofs": dofs},
            "cpu_baseline": full,
            "e2e": {"value": v, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    from oracle.krylov import pcg
    sample = _oracle_sample()
    dofs = sum(s[1] for s in sample)
    t_tot, steps = 0.0, 0
    while True:
        t0 = time.time()
        for (_, _, A, M, b) in sample:
            _, info = pcg(A, b, M.apply, rtol=1e-8, flexible=True)
        t_tot += time.time() - t0
        steps += 1
        if t_tot > budget_s / 3 or steps >= 3:
            break
    return {"value": steps * dofs / t_tot, "unit": "DOFs/s", "cores": cores, "kind": "oracle",
            "same_config": False,
            "sample": f"oracle PCG solves (setup excluded) of the same H(grad)+H(curl) problems "
                      f"on a 3x3x3 mesh, p={DEGREE} ({dofs} lattice DOFs), {steps} step(s)"}


def oracle_full_worker(cache):
    """The oracle's solves of the whole workload (8x8x8 mesh, p = 7, both
    spaces): setup timed apart from the solve; one JSON line.  The set-up
    problems (operator, preconditioner, right-hand side) are pickled to
    `cache` by the first run and loaded by later ones."""
    import pickle
    from oracle.auxiliary import assemble_aux
    from oracle.discretization import Problem
    from oracle.krylov import pcg
    from oracle.relaxation import SCPAFW, SCPH
    from paper_2211_14284_gb300 import inputs
    n = N_CELLS
    out = {"dofs": 0, "setup_s": 0.0, "solve_s": 0.0, "iterations": {}, "setup_cached": False}
    for sname, k, _ in SPACES:
        path = os.path.join(cache, f"oracle_{sname}.pickle")
        t0 = time.time()
        if os.path.exists(path):
            with open(path, "rb") as f:
                size, A, M, b = pickle.load(f)
            out["setup_cached"] = True
        else:
            X = inputs.vertices(n, perturb=PERTURB, seed=2)
            al = inputs.constant_coefficient(n)
            be = inputs.constant_coefficient(n)
            pr = Problem(k, n, DEGREE, X, al, be)
            A = pr.A_free()
            P = assemble_aux(pr)[pr.free][:, pr.free]
            M = SCPAFW(pr, P, factor="icc") if k == 0 else SCPH(pr, P)
            b = inputs.normal_rhs(pr.lat.size, 100 + k)[pr.free]
            size = pr.lat.size
            with open(path, "wb") as f:
                pickle.dump((size, A, M, b), f, protocol=pickle.HIGHEST_PROTOCOL)
        t1 = time.time()
        _, info = pcg(A, b, M.apply, rtol=1e-8, flexible=True)
        t2 = time.time()
        out["dofs"] += size
        out["setup_s"] += t1 - t0
        out["solve_s"] += t2 - t1
        out["iterations"][sname] = info["iterations"]
    print(json.dumps(out))


def cpu_baseline_full():
    """The oracle on the full workload, with BLAS/OpenMP threads on every
    core of this host and single-threaded (each in its own process; the
    second loads the first one's set-up from a scratch directory)."""
    cores = len(os.sched_getaffinity(0))
    res = {}
    with tempfile.TemporaryDirectory() as cache:
        for label, th in (("all_cores", cores), ("1_thread", 1)):
            env = dict(os.environ)
            for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                env[v] = str(th)
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-full-worker", cache],
                               capture_output=True, text=True, env=env)
            if r.returncode != 0:
                raise RuntimeError(r.stderr[-2000:])
            d = json.loads(r.stdout.strip().splitlines()[-1])
            d["value"] = d["dofs"] / d["solve_s"]
            d["threads"] = th
            res[label] = d
    return {"value": res["all_cores"]["value"], "unit": "DOFs/s", "cores": cores, "kind": "oracle",
            "same_config": True, "runs": res,
            "sample": f"the whole workload (8x8x8, p={DEGREE}, H(grad)+H(curl)), setup excluded"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    if args.cpu_baseline_full:
        # the whole workload (one solve per space, set-up excluded), minutes
        full = cpu_baseline_full()
        v = full["value"]
        dofs = full["runs"]["all_cores"]["dofs"]
        print(json.dumps({
            "metric": METRIC, "value": v, "unit": "DOFs/s", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * dofs / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice_dofs": dofs},
            "cpu_baseline": full,
            "e2e": {"value": v, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    from oracle.krylov import pcg
    sample = _oracle_sample()
    dofs = sum(s[1] for s in sample)

    def step():
        for (_, _, A, M, b) in sample:
            pcg(A, b, M.apply, rtol=1e-8, flexible=True)

    for _ in range(args.warmup):
        step()
    t0 = time.time()
    for _ in range(args.steps):
        step()
    dt = time.time() - t0
    v = args.steps * dofs / dt
    line = {
        "metric": METRIC, "value": v, "unit": "DOFs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": WORKLOAD + " (oracle sample: 3x3x3 mesh)", "lattice_dofs": dofs},
        "cpu_baseline": {"value": v, "unit": "DOFs/s", "cores": cores, "kind": "oracle",
                         "sample": f"3x3x3 mesh, p={DEGREE}, H(grad)+H(curl), {dofs} lattice DOFs"},
        "e2e": {"value": v, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def batched_problems(count):
    """The uneven H(curl) batch (n ~ U{4..12}, p ~ U{3..12}, beta log-uniform
    in [0.1, 10], alpha = 1); count < 64 takes the first `count` problems with
    n, p <= 8 (a bounded sample whose host setup stays short)."""
    from paper_2211_14284_gb300 import inputs
    probs = inputs.batched_hcurl_problems(64, seed=4)
    if count < 64:
        probs = [p for p in probs if p["n"] <= 8 and p["p"] <= 8][:count]
    out = []
    for pr in probs:
        nc = pr["n"] ** 3
        out.append({"space": 1, "n": pr["n"], "p": pr["p"], "alpha": [pr["alpha"]] * nc,
                    "beta": [pr["beta"]] * nc, "rhs_seed": pr["rhs_seed"]})
    return out


def run_batched(count, steps, warmup, stream):
    """Uneven H(curl) problems: the batched solver (one graph-captured
    lock-step iteration for all) against solving them one after another with
    the single-problem solver; SC-PH, ICC(0) potential patches, P1 coarse."""
    import torch
    from paper_2211_14284_gb300 import inputs
    from paper_2211_14284_gb300.rm import BatchSolver, Solver
    probs = batched_problems(count)
    opts = dict(static_condensation=1, decomposition=1, factor=1, rtol=1e-8, max_it=1000)
    t0 = time.time()
    B = BatchSolver(probs, check_every=8, **opts)
    setup_s = time.time() - t0
    singles = [Solver(1, pr["n"], pr["p"], alpha=pr["alpha"], beta=pr["beta"], stream=stream, **opts)
               for pr in probs]
    bs = [torch.tensor(inputs.normal_rhs(sz, pr["rhs_seed"]), device="cuda")
          for pr, sz in zip(probs, B.sizes)]
    xs = [torch.zeros_like(b) for b in bs]
    dofs = sum(B.sizes)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def time_it(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            for x in xs:
                x.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            out = fn()
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
        return tot / steps, out

    def batched():
        infos = B.solve(bs, xs, stream=stream)
        if not all(i["status"] == "RM_OK" for i in infos):
            raise RuntimeError("batched solve did not converge")
        return infos

    def sequential():
        infos = [s.solve(b, x) for s, b, x in zip(singles, bs, xs)]
        if not all(i["status"] == "RM_OK" for i in infos):
            raise RuntimeError("sequential solve did not converge")
        return infos

    ms_b, ib = time_it(batched)
    ms_s, isq = time_it(sequential)
    return {"problems": len(probs), "lattice_dofs": dofs, "setup_s": setup_s,
            "value": dofs / (ms_b / 1e3), "ms_per_step": ms_b,
            "sequential_value": dofs / (ms_s / 1e3), "sequential_ms_per_step": ms_s,
            "speedup_vs_sequential": ms_s / ms_b,
            "iterations_max": max(i["iterations"] for i in ib),
            "kernel_launches_per_solve": ib[0]["kernel_launches"],
            "sample": ("all 64 problems" if count >= 64 else
                       f"first {len(probs)} problems with n, p <= 8")}


def run_learned(steps, warmup, epochs, n, stream, on_policy_rounds=2):
    """H(grad) on n^3 (default 32^3) uniform cells, p = 6, lognormal Gaussian-random-field
    alpha: the learned coarse corrector (trained here on pairs the solver
    generates) against the plain coarse correction (the V(2,2) cycle) and
    against no coarse term; SC-PAFW with ICC(0) patches."""
    import torch
    from paper_2211_14284_gb300 import inputs
    from paper_2211_14284_gb300.rm import (RM_CORRECTOR_LEARNED, RM_CORRECTOR_OFF,
                                           RM_CORRECTOR_PLAIN, Solver)
    p = 6
    al = inputs.lognormal_grf_coefficient(n, 1.0, 0.1, seed=5)
    t0 = time.time()
    s = Solver(0, n, p, alpha=al, stream=stream, static_condensation=1, factor=1, coarse=2,
               rtol=1e-8, max_it=1000)
    setup_s = time.time() - t0
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20221125)
    rhs = torch.randn(150, s.size, dtype=torch.float64, device="cuda", generator=gen)
    train = s.corrector_train(rhs, pairs=2000, epochs=epochs, levels=3, width=16, batch=16,
                              lr=2e-3)
    b = torch.tensor(inputs.normal_rhs(s.size, 77), device="cuda")
    x = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def time_mode(mode, every, jmax, nsteps, nwarm):
        s.corrector_use(mode, every, jmax)
        for _ in range(nwarm):
            x.zero_()
            s.solve(b, x)
        torch.cuda.synchronize()
        tot, info = 0.0, None
        for _ in range(nsteps):
            flush.fill_(1.0)
            x.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            info = s.solve(b, x)
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
            if info["status"] != "RM_OK":
                raise RuntimeError(f"learned-corrector bench: {info}")
        ms = tot / nsteps
        return {"value": s.size / (ms / 1e3), "ms_per_solve": ms, "iterations": info["iterations"],
                "learned_calls": info["learned_calls"], "judge_calls": info["judge_calls"],
                "fallback_at": info["fallback_at"], "judge_eta": info["judge_eta"]}

    out = {"workload": f"H(grad), {n}^3 uniform hex, p=6, lognormal GRF alpha (sigma 1, "
                       "ell 0.1), beta=1, SC-PAFW + ICC, V(2,2) coarse cycle",
           "lattice_dofs": s.size, "setup_s": setup_s, "train": train,
           "plain": time_mode(RM_CORRECTOR_PLAIN, 0, 1.0, steps, warmup),
           "learned": time_mode(RM_CORRECTOR_LEARNED, 4, 0.9, steps, warmup),
           "learned_unjudged": time_mode(RM_CORRECTOR_LEARNED, 0, 1.0, 1, 0),
           "off": time_mode(RM_CORRECTOR_OFF, 0, 1.0, 1, 0)}
    # on-policy: two more rounds of pairs from solves that use the network
    if on_policy_rounds > 0:
        s.corrector_use(RM_CORRECTOR_PLAIN, 0, 1.0)
        out["train_on_policy"] = s.corrector_train(rhs, pairs=2000, epochs=epochs, levels=3, width=16,
                                                   batch=16, lr=2e-3, rounds=on_policy_rounds,
                                                   round_pairs=500, round_epochs=max(1, epochs // 2))
        out["learned_on_policy"] = time_mode(RM_CORRECTOR_LEARNED, 4, 0.9, steps, warmup)
        out["learned_on_policy_unjudged"] = time_mode(RM_CORRECTOR_LEARNED, 0, 1.0, 1, 0)
    del rhs
    s.corrector_use(RM_CORRECTOR_PLAIN, 0, 1.0)
    out["value"] = out["learned"]["value"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-full", action="store_true",
                    help="time the oracle on the whole workload (minutes of host setup) instead of a sample")
    ap.add_argument("--oracle-full-worker", metavar="CACHE_DIR", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-apply-kernels", action="store_true",
                    help="skip timing the Cartesian operator apply on its own workloads")
    ap.add_argument("--deterministic", action="store_true",
                    help="bitwise-reproducible relaxation (rm_options.deterministic = 1) in every variant")
    ap.add_argument("--sequential", action="store_true",
                    help="solve the two problems of a step one after another on one host thread "
                         "(for profilers, which serialise kernels anyway)")
    ap.add_argument("--batch-count", type=int, default=8,
                    help="problems of the uneven H(curl) batch to time (64 = all; 0 = skip)")
    ap.add_argument("--learned-size", type=int, default=32,
                    help="cells per direction of the learned-corrector workload (multiple of 8)")
    ap.add_argument("--learned-epochs", type=int, default=10,
                    help="training epochs of the learned coarse corrector (0 = skip that variant)")
    args = ap.parse_args()
    if args.oracle_full_worker:
        oracle_full_worker(args.oracle_full_worker)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
