"""Benchmark: one step = one SRJ solve of the 2D Poisson problem on a
4096 x 4096 interior grid (5-point stencil, zero Dirichlet, f i.i.d.
uniform[-1, 1] seed 0, u0 = 0) to relative residual 1e-8, with the paper's
scheme family and Alg. 1 selection, through the library's C ABI.

The timed solve is the mixed-precision path (FP64 refinement around
FP32-arithmetic inner SRJ on an FP32-pair iterate); the plain FP64 SRJ solve
of the same problem is timed once afterwards for the mixed-vs-plain ratio.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (the
solve does not shard across GPUs here): each rank solves its own seeded
problem, value = all ranks' grid-point updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("GLUP/s (% HBM roofline) and time to 1e-8 rel. residual, learned/mixed vs plain SRJ")
UNIT = "GLUP/s"
SIDE = 4096
TOL = 1e-8
# FP32 instructions per grid-point update of the FP32-pair relaxation of the
# isotropic 2D workload (df_pair_sum + df_relax_iso_pairs in csrc/df32.cuh):
# the shared diagonal pair sum (8), the second pair sum (8), q = s/4 + g as an
# error-free sum (6 + 1), the two products (1 - omega) u and omega q with
# their errors (6), their error-free sum (6), two low-part adds and one Dekker
# renormalisation (5).
DF_OPS_PER_LUP = 40  # FP32 instructions per update of the fused isotropic FP32-pair form
# algorithmic HBM bytes of an FP32 sweep per grid point and pass: read u, read
# f, write u (4 B each); 3D variable coefficients add k (4 B)
ALGO_BYTES_PER_POINT = 12.0
ALGO_BYTES_PER_POINT_VARK = 16.0
WORKLOAD = ("2D Poisson 5-point, 4096x4096 interior, zero Dirichlet, f~U[-1,1] (seed 0+rank), "
            "u0=0, rel residual 1e-8, SRJ scheme family + Alg. 1 heuristic")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# sources of the dominant kernel (FP32-pair wave pass); the DRAM traffic taken
# from an ncu capture is reported only while these files are unchanged
KERNEL_SOURCES = ["paper_2011_06636_gb300/csrc/" + f for f in (
    "wave_item.cuh", "kernels_wave2d.cu", "df32.cuh", "stencil_point.cuh", "pass_common.cuh",
    "mlp.cuh", "srj_internal.h")]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "wave2d_fp32pair_T2_4096.md")


# the same for the 3D mixed solve's pass (captured at 256^3: its traffic is
# scaled to the bench's grid by the points of a launch)
KERNEL_SOURCES_3D = ["paper_2011_06636_gb300/csrc/" + f for f in (
    "kernels_plane3d.cu", "df32.cuh", "df32x2.cuh", "stencil_point.cuh", "pass_common.cuh",
    "mlp.cuh", "srj_internal.h")]
PROFILE_SUMMARY_3D = os.path.join(ROOT, "profiles", "plane3d2_fp32pair_vark_256.md")
PROFILE_POINTS_3D = 256 ** 3


def kernel_source_hash(sources=KERNEL_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(summary=PROFILE_SUMMARY, sources=KERNEL_SOURCES):
    """DRAM bytes per launch of a kernel from its committed ncu summary, or
    None when it is absent or the kernel's sources changed since."""
    if not os.path.exists(summary):
        return None
    vals = {}
    for line in open(summary):
        if ":" in line and line.strip().startswith(("dram_bytes_per_launch", "source_sha256")):
            k, v = line.strip().split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != kernel_source_hash(sources):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def fp32_issue_peak(sm_mhz):
    """FP32 instruction rate of the GPU: 152 SMs x 128 FP32 lanes x clock
    (one instruction per lane per cycle, FMA counted once), in T instr/s."""
    return 152 * 128 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SRJ_BENCH_GLOO") is None else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(world, v, op):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allmax(world, v):
    import torch.distributed as dist
    return _reduce(world, v, dist.ReduceOp.MAX if world > 1 else None)


def allsum(world, v):
    import torch.distributed as dist
    return _reduce(world, v, dist.ReduceOp.SUM if world > 1 else None)


def replica_throughput(world, lups_local, ms_local):
    """Whole-job throughput of independent replicas: every rank's grid-point
    updates over the slowest rank's time.  Returns (GLUP/s, max ms)."""
    ms_max = allmax(world, ms_local)
    lups = allsum(world, float(lups_local))
    return lups / (ms_max * 1e-3) / 1e9, ms_max


# ----------------------------------------------------------------- oracle arm
def host_cores():
    """Host cores this process may run on (the OpenMP oracle's thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(seconds_budget=15.0, parallel=False):
    """Time the FP64 oracle's sweeps on the same 4096^2 problem: whole cycles
    at levels 0, 1, 2, ... until the budget is used; parallel=True runs the
    OpenMP build of the same source on all host cores.  Returns (GLUP/s,
    seconds, text, threads)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2011_06636_gb300 import inputs
    n = [SIDE, SIDE]
    f = inputs.uniform_rhs(n, seed=0).ravel()
    P = O.Problem(n)
    u = np.zeros(f.size)
    threads = 1
    if parallel:
        threads = int(os.environ.get("OMP_NUM_THREADS", host_cores()))
        O.omp_lib()
    t0 = time.perf_counter()
    sweeps, level = 0, 0
    while True:
        w = O.level_omegas(level)
        u = O.sweeps(P, u, f, w, parallel=parallel)
        sweeps += len(w)
        level += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    dt = time.perf_counter() - t0
    text = "%d sweeps (cycles at levels 0..%d) of the 4096^2 problem, %d thread%s" % (
        sweeps, level - 1, threads, "" if threads == 1 else "s")
    return sweeps * f.size / dt / 1e9, dt, text, threads


def cpu_baseline_line(seconds_all, seconds_one):
    """The oracle on all host cores (the reported baseline) and on one core."""
    try:
        v, _, sample, threads = oracle_sample(seconds_all, parallel=True)
    except (OSError, subprocess.CalledProcessError) as e:  # no OpenMP toolchain
        v, _, sample, threads = oracle_sample(seconds_all)
        sample += " (OpenMP build unavailable: %s)" % str(e).splitlines()[0][:80]
    out = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
    if seconds_one > 0:
        v1, _, s1, _ = oracle_sample(seconds_one)
        out["single_core"] = {"value": v1, "unit": UNIT, "cores": 1, "sample": s1}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    budget = float(os.environ.get("SRJ_ORACLE_STEP_SECONDS", "6"))
    try:
        O.build_omp()
        parallel = True
    except (OSError, subprocess.CalledProcessError):
        parallel = False
    for _ in range(args.warmup):
        oracle_sample(budget / 4, parallel=parallel)
    vals, times, sample, threads = [], [], "", 1
    for _ in range(args.steps):
        v, dt, sample, threads = oracle_sample(budget, parallel=parallel)
        vals.append(v)
        times.append(dt)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [SIDE, SIDE]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "each step: " + sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched
def batched_leg(srj, inputs, torch, stream, seed=0, count=256, fp64=True):
    """256 independent 2D problems (sides U{64..1024}, half anisotropic), f ~
    N(0,1), rel 1e-8: one batched mixed-precision solve (persistent kernel in
    a CUDA graph, autotuned depth/segment), against the same problems solved
    one after another on the same GPU by the single-grid mixed-precision solve
    and by plain FP64 SRJ with Alg. 1 (the second solve of each handle)."""
    probs = inputs.batched_problems(count=count, seed=seed)
    ns = [p["n"] for p in probs]
    eps = [p["eps"] for p in probs]
    fs = [torch.as_tensor(inputs.normal_rhs(p["n"], seed=p["seed_f"]).ravel(), device="cuda")
          for p in probs]
    us = [torch.zeros_like(f) for f in fs]
    npts = [f.numel() for f in fs]
    h = srj.srj_create_batched(ns, eps=eps, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    rc, st = srj.srj_solve_batched(h, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], TOL)
    tune_s = time.perf_counter() - t0  # first call includes the autotuner
    for u in us:
        u.zero_()
    rc, st = srj.srj_solve_batched(h, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], TOL)
    srj.srj_destroy(h)
    mlp = None
    from paper_2011_06636_gb300 import selector
    if os.path.exists(selector.WEIGHTS):
        hm = srj.srj_create_batched(ns, eps=eps, selector=srj.SRJ_SEL_MLP,
                                    stream=stream.cuda_stream)
        srj.srj_mlp_set_weights(hm, selector.load_weights())
        for u in us:
            u.zero_()
        srj.srj_solve_batched(hm, [f.data_ptr() for f in fs], [u.data_ptr() for u in us], TOL)
        for u in us:
            u.zero_()
        rcm, stm = srj.srj_solve_batched(hm, [f.data_ptr() for f in fs],
                                         [u.data_ptr() for u in us], TOL)
        srj.srj_destroy(hm)
        mlp = {"time_to_tol_s": stm[0]["seconds"], "converged": rcm == srj.SRJ_OK,
               "sweeps_total": sum(x["sweeps"] for x in stm)}
    secs = st[0]["seconds"]
    lups = sum(s["sweeps"] * n for s, n in zip(st, npts))
    out = {"problems": count, "points": sum(npts), "converged": rc == srj.SRJ_OK,
           "time_to_tol_s": secs, "glups": lups / secs / 1e9,
           "sweeps_total": sum(s["sweeps"] for s in st), "first_call_with_autotune_s": tune_s,
           "learned_selector": mlp}
    # the same problems one after another through the single-grid
    # mixed-precision solve (the batched kernel's own engine, one problem at
    # a time); each handle's first solve builds its graph, the second is timed
    tot, lups1, ok = 0.0, 0.0, True
    for p, f in zip(probs, fs):
        h1 = srj.srj_create(p["n"], eps=p["eps"], precision=srj.SRJ_PREC_MIXED,
                            stream=stream.cuda_stream)
        u = torch.zeros_like(f)
        srj.srj_solve(h1, f.data_ptr(), u.data_ptr(), TOL)
        u.zero_()
        s1 = srj.srj_solve(h1, f.data_ptr(), u.data_ptr(), TOL)
        srj.srj_destroy(h1)
        tot += s1["seconds"]
        lups1 += s1["sweeps"] * f.numel()
        ok = ok and s1["status"] == srj.SRJ_OK
    out["mixed_sequential"] = {"time_to_tol_s": tot, "glups": lups1 / tot / 1e9,
                               "converged": ok}
    out["speedup_vs_mixed_sequential"] = tot / secs
    if fp64:
        tot, sw64, ok = 0.0, 0, True
        for p, f in zip(probs, fs):
            h64 = srj.srj_create(p["n"], eps=p["eps"], precision=srj.SRJ_PREC_F64,
                                 stream=stream.cuda_stream)
            u = torch.zeros_like(f)
            srj.srj_solve(h64, f.data_ptr(), u.data_ptr(), TOL)  # builds the graph
            u.zero_()
            s64 = srj.srj_solve(h64, f.data_ptr(), u.data_ptr(), TOL)
            srj.srj_destroy(h64)
            tot += s64["seconds"]
            sw64 += s64["sweeps"]
            ok = ok and s64["status"] == srj.SRJ_OK
        out["plain_fp64_sequential"] = {"time_to_tol_s": tot, "sweeps_total": sw64, "converged": ok}
        out["speedup_vs_plain_fp64"] = tot / secs
        if mlp:
            out["learned_selector"]["speedup_vs_plain_fp64"] = tot / mlp["time_to_tol_s"]
    return out


# ------------------------------------------------------------------- multigrid
def mg_leg(srj, inputs, torch, stream, seed=0, side=4095):
    """Multigrid with SRJ smoothing on the 2D Poisson problem of the headline
    (4095^2: n = 2^k - 1 for the hierarchy), f ~ U[-1,1], rel 1e-8, FP64:
    the SRJ level-1 smoother (M = 2) and the classic damped Jacobi (level 0,
    omega = 2/3), both V(1,1)."""
    n = [side, side]
    f = torch.as_tensor(inputs.uniform_rhs(n, seed=seed).ravel(), device="cuda")
    out = {"grid": n, "tol": TOL}
    for label, lv in (("srj_level1_smoother", 1), ("damped_jacobi_smoother", 0)):
        h = srj.srj_mg_create(n, smoother_level=lv, stream=stream.cuda_stream)
        u = torch.zeros_like(f)
        srj.srj_mg_solve(h, f.data_ptr(), u.data_ptr(), TOL)  # warm-up (graph capture)
        u.zero_()
        st = srj.srj_mg_solve(h, f.data_ptr(), u.data_ptr(), TOL)
        srj.srj_destroy(h)
        out[label] = {"time_to_tol_s": st["seconds"], "vcycles": st["cycles"],
                      "fine_sweeps": st["sweeps"], "kernel_launches": st["passes"],
                      "rel_residual": st["rn"] / st["r0"],
                      "status": srj.STATUS_NAMES[st["status"]]}
    return out


# -------------------------------------------------------- the paper's studies
def paper_studies_leg(srj, inputs, torch, stream, seed=0):
    """Two of the paper's out-of-sample studies, timed on the GPU (FP64, the
    paper's own stopping rules; sweep counts are the ones the parity tests
    compare with the oracle):
      * Sec. 4.1: random symmetric diagonally dominant tridiagonal systems,
        N = 10, 100, 500, 1000, 20 matrices each (seeds 0..19), b = 1,
        x0 = 0, ||b - A x||_2 < 1e-7; Alg. 1 against the increasing rule;
      * Sec. 4.2.2: 2D Laplace with homogeneous Neumann boundaries, the
        paper's size sweep 32^2 ... 1024^2 nodes, 10 random starts U[-1,1]
        each, ||x^n - x^(n-1)||_inf < 1e-10 tested after every sweep; Alg. 1
        against the increasing rule, and the sizes where the ranking holds."""
    rules = (("heuristic", srj.SRJ_SEL_HEURISTIC), ("increasing", srj.SRJ_SEL_INCREASING))
    tri = {}
    for N in (10, 100, 500, 1000):
        row = {}
        for label, sel in rules:
            sw, secs, ok = [], [], True
            for m in range(20):
                d, e = inputs.random_sdd_tridiagonal(N, seed=m)
                ad = torch.as_tensor(d, device="cuda")
                ao = torch.as_tensor(e, device="cuda")
                h = srj.srj_create([N], precision=srj.SRJ_PREC_F64, tol_kind=srj.SRJ_TOL_ABS,
                                   selector=sel, stream=stream.cuda_stream,
                                   a_diag_ptr=ad.data_ptr(), a_off_ptrs=[ao.data_ptr()])
                f = torch.ones(N, dtype=torch.float64, device="cuda")
                u = torch.zeros_like(f)
                st = srj.srj_solve(h, f.data_ptr(), u.data_ptr(), 1e-7)
                srj.srj_destroy(h)
                sw.append(st["sweeps"])
                secs.append(st["seconds"])
                ok = ok and st["status"] == srj.SRJ_OK
            row[label] = {"mean_sweeps": sum(sw) / len(sw), "mean_solve_ms": 1e3 * sum(secs) / len(secs),
                          "all_converged": ok}
        row["increasing_over_heuristic"] = (row["increasing"]["mean_sweeps"]
                                            / row["heuristic"]["mean_sweeps"])
        tri["N=%d" % N] = row
    lap = {}
    for side in (32, 64, 128, 256, 512, 1024):
        n = [side, side]
        f = torch.zeros(side * side, dtype=torch.float64, device="cuda")
        row = {}
        for label, sel in rules:
            h = srj.srj_create(n, bc=[srj.SRJ_BC_NEUMANN] * 2, precision=srj.SRJ_PREC_F64,
                               tol_kind=srj.SRJ_TOL_DINF, selector=sel, stream=stream.cuda_stream)
            sw, secs, ok = [], [], True
            for trial in range(10):
                u = torch.as_tensor(inputs.uniform_rhs(n, seed=seed + trial).ravel(), device="cuda")
                st = srj.srj_solve(h, f.data_ptr(), u.data_ptr(), 1e-10)
                sw.append(st["sweeps"])
                secs.append(st["seconds"])
                ok = ok and st["status"] == srj.SRJ_OK
            srj.srj_destroy(h)
            mean_s = sum(secs) / len(secs)
            row[label] = {"mean_sweeps": sum(sw) / len(sw), "mean_solve_s": mean_s,
                          "glups": sum(sw) * side * side / sum(secs) / 1e9, "all_converged": ok}
        row["heuristic_fewer_sweeps"] = row["heuristic"]["mean_sweeps"] < row["increasing"]["mean_sweeps"]
        lap["%dx%d" % (side, side)] = row
    return {"random_tridiagonal_sec4_1": tri, "laplace_neumann_sec4_2_2": lap}


# ----------------------------------------------------------- learned selector
def selector_leg(srj, inputs, torch, stream, seed=0):
    """Unseen problems for the learned selector: 2D anisotropic (eps_x = 0.01)
    at 2048^2 and 3D log-normal variable-coefficient diffusion at 256^3, both
    f ~ N(0,1), rel 1e-8, mixed precision; Alg. 1 vs the network (with Alg. 1
    as fallback) on the same GPU."""
    from paper_2011_06636_gb300 import selector
    if not os.path.exists(selector.WEIGHTS):
        return {"unavailable": "no trained selector weights (selector_bf16.bin)"}
    w = selector.load_weights()
    cases = [("2d_aniso_eps0.01_2048", [2048, 2048], [0.01, 1.0], None),
             ("3d_lognormal_k_256", [256, 256, 256], None, "k")]
    out = {}
    for name, n, eps, kind in cases:
        f = torch.as_tensor(inputs.normal_rhs(n, seed=seed + 7).ravel(), device="cuda")
        kt = None
        if kind:
            kt = torch.as_tensor(inputs.lognormal_k(n, seed=seed + 8).ravel(), device="cuda")
        res = {}
        for label, sel, prec in (("heuristic", srj.SRJ_SEL_HEURISTIC, srj.SRJ_PREC_MIXED),
                                 ("mlp", srj.SRJ_SEL_MLP, srj.SRJ_PREC_MIXED),
                                 ("plain_fp64_heuristic", srj.SRJ_SEL_HEURISTIC,
                                  srj.SRJ_PREC_F64)):
            h = srj.srj_create(n, eps=eps, k_ptr=kt.data_ptr() if kt is not None else None,
                               selector=sel, precision=prec, stream=stream.cuda_stream)
            if sel == srj.SRJ_SEL_MLP:
                srj.srj_mlp_set_weights(h, w)
            u = torch.zeros_like(f)
            srj.srj_solve(h, f.data_ptr(), u.data_ptr(), TOL)  # warm-up (graph build)
            u.zero_()
            st = srj.srj_solve(h, f.data_ptr(), u.data_ptr(), TOL)
            srj.srj_destroy(h)
            res[label] = {"time_to_tol_s": st["seconds"], "cycles": st["cycles"],
                          "sweeps": st["sweeps"], "outer": st["outer"],
                          "status": srj.STATUS_NAMES[st["status"]]}
        res["mlp_vs_heuristic_speedup"] = (res["heuristic"]["time_to_tol_s"] /
                                           res["mlp"]["time_to_tol_s"])
        res["mlp_mixed_vs_plain_fp64_speedup"] = (res["plain_fp64_heuristic"]["time_to_tol_s"] /
                                                  res["mlp"]["time_to_tol_s"])
        out[name] = res
    return out


def vark3d_leg(srj, inputs, torch, stream, seed=0, side=512, fp64=True, depth=0):
    """3D variable-coefficient diffusion -div(k grad u) = f, 7-point stencil,
    harmonic-mean faces, log k Gaussian random field (correlation 16 cells,
    sigma 1), f ~ N(0,1), rel 1e-8: mixed precision (FP32-pair inner SRJ
    inside FP64 refinement) vs plain FP64 SRJ on the same GPU, with the
    relative difference of the two solutions."""
    n = [side] * 3
    f = torch.as_tensor(inputs.normal_rhs(n, seed=seed + 3).ravel(), device="cuda")
    kt = torch.as_tensor(inputs.lognormal_k(n, seed=seed + 4).ravel(), device="cuda")
    res = {}
    sols = {}
    for label, prec in (("mixed", srj.SRJ_PREC_MIXED), ("plain_fp64", srj.SRJ_PREC_F64)):
        if label == "plain_fp64" and not fp64:
            continue
        h = srj.srj_create(n, k_ptr=kt.data_ptr(), precision=prec, stream=stream.cuda_stream,
                           temporal_depth=depth if label == "mixed" else 0)
        u = torch.zeros_like(f)
        st = srj.srj_solve(h, f.data_ptr(), u.data_ptr(), TOL)
        srj.srj_destroy(h)
        res[label] = {"time_to_tol_s": st["seconds"], "sweeps": st["sweeps"],
                      "cycles": st["cycles"], "outer": st["outer"],
                      "glups": st["sweeps"] * f.numel() / st["seconds"] / 1e9,
                      "rel_residual": st["rn"] / st["r0"],
                      "status": srj.STATUS_NAMES[st["status"]]}
        if label == "mixed":
            # roofline of the inner passes (plane3d2_kernel, two sweeps per
            # pass): algorithmic 16 B per update (read u, r, k; write u,
            # FP32), over the device time of the inner cycle loops; the
            # FP32-pair design moves 36 B per point and pass (iterate hi/lo
            # read and write 16, rhs 4, three face weights and 1/D 16), 18 B
            # per update with two sweeps per pass
            hbm_peak, peak_kind = peaks()
            inner_s = st["inner_seconds"]
            ach = ALGO_BYTES_PER_POINT_VARK * st["sweeps"] * f.numel() / inner_s / 1e9
            res[label]["inner_seconds"] = inner_s
            tr = profiled_traffic(PROFILE_SUMMARY_3D, KERNEL_SOURCES_3D)
            res[label]["roofline"] = {
                "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak,
                "traffic": tr * f.numel() / PROFILE_POINTS_3D if tr else None,
                "traffic_note": "ncu DRAM bytes of one two-sweep launch at 256^3, scaled to "
                                "this grid by its points",
                "kernel": "plane3d2_kernel<FP32-pair, variable k> (two sweeps per pass)",
                "algorithmic_bytes_per_update": ALGO_BYTES_PER_POINT_VARK,
                "bytes_moved_per_update_by_design": 18.0,
                "design_bytes_frac": 18.0 * st["sweeps"] * f.numel() / inner_s / 1e9 / hbm_peak,
                "timing": "CUDA events around the inner cycle loops",
                "peak_kind": peak_kind}
        sols[label] = u
    if "plain_fp64" in sols:
        d = torch.linalg.norm(sols["mixed"] - sols["plain_fp64"]) / torch.linalg.norm(
            sols["plain_fp64"])
        res["mixed_vs_fp64_rel_solution_diff"] = float(d)
        res["speedup"] = res["plain_fp64"]["time_to_tol_s"] / res["mixed"]["time_to_tol_s"]
    return res


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_2011_06636_gb300 import _build, inputs, srj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    _build.build()
    srj.load(build_if_missing=False)
    side = args.side
    n = [side, side]
    npts = side * side
    f_np = inputs.uniform_rhs(n, seed=rank).ravel()
    stream = torch.cuda.current_stream()
    f = torch.as_tensor(f_np, device="cuda")
    u = torch.zeros(npts, dtype=torch.float64, device="cuda")
    h = srj.srj_create(n, precision=srj.SRJ_PREC_MIXED, stream=stream.cuda_stream,
                       temporal_depth=args.depth)

    def step():
        u.zero_()
        return srj.srj_solve(h, f.data_ptr(), u.data_ptr(), TOL)

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()
    barrier(world)
    stats = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        ev0.record(stream)
        for _ in range(args.steps):
            stats.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    sweeps = sum(s["sweeps"] for s in stats)
    passes = sum(s["passes"] for s in stats)
    outer = sum(s["outer"] for s in stats)
    value, ms_max = replica_throughput(world, float(sweeps) * npts, ms)
    ok = all(s["status"] == srj.SRJ_OK for s in stats)
    # relative residual of the last solve, checked independently in FP64 torch
    uu = u.view(side, side)
    ff = f.view(side, side)
    up = torch.nn.functional.pad(uu, (1, 1, 1, 1))
    hinv2 = float((side + 1) ** 2)
    Au = hinv2 * (4 * uu - up[1:-1, :-2] - up[1:-1, 2:] - up[:-2, 1:-1] - up[2:, 1:-1])
    rel_check = float(torch.linalg.norm(ff - Au) / torch.linalg.norm(ff))

    # dominant kernel: the inner pass.  Its average launch duration is the
    # device time of the cycle loops (CUDA events around each inner solve's
    # loop on the library's stream, so without the outer FP64 kernels) over
    # the passes they ran.
    clocks = clk.summary()
    inner_s = sum(s["inner_seconds"] for s in stats)
    pass_s = inner_s / max(passes, 1)
    sweeps_per_pass = sweeps / max(passes, 1)
    hbm_peak, peak_kind = peaks()
    # algorithmic bytes of the FP32 inner sweep: read u, read f, write u,
    # 4 B each per grid point and HBM pass; effective: per update
    algo_per_pass = ALGO_BYTES_PER_POINT * npts
    hbm_achieved = algo_per_pass / pass_s / 1e9
    hbm_effective = ALGO_BYTES_PER_POINT * sweeps * npts / inner_s / 1e9
    moved_per_pass = 20.0 * npts  # what the FP32-pair design moves: hi, lo read+write, rhs
    sm_mhz = clocks["sm_mhz"] or 2070.0
    alu_peak = fp32_issue_peak(sm_mhz)
    alu_achieved = DF_OPS_PER_LUP * npts * sweeps_per_pass / pass_s / 1e12

    # end to end through srj_solve_host with pinned host buffers
    e2e_val = None
    if not args.no_e2e:
        fh = torch.as_tensor(f_np).pin_memory()
        uh = torch.zeros(npts, dtype=torch.float64).pin_memory()
        e2e_st = srj.srj_solve_host(h, fh.data_ptr(), uh.data_ptr(), TOL)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        e2e_sweeps = 0
        for _ in range(args.steps):
            uh.zero_()
            e2e_st = srj.srj_solve_host(h, fh.data_ptr(), uh.data_ptr(), TOL)
            e2e_sweeps += e2e_st["sweeps"]
        e2e_s = allmax(world, time.perf_counter() - t0)
        e2e_val = allsum(world, float(e2e_sweeps) * npts) / e2e_s / 1e9
    srj.srj_destroy(h)

    # plain FP64 SRJ with the heuristic on the same problem (comparator)
    fp64 = None
    if not args.no_fp64:
        h64 = srj.srj_create(n, precision=srj.SRJ_PREC_F64, stream=stream.cuda_stream)
        u.zero_()
        s64 = srj.srj_solve(h64, f.data_ptr(), u.data_ptr(), TOL)
        srj.srj_destroy(h64)
        fp64 = {"time_to_tol_s": s64["seconds"], "sweeps": s64["sweeps"],
                "glups": s64["sweeps"] * npts / s64["seconds"] / 1e9,
                "status": srj.STATUS_NAMES[s64["status"]]}

    # FP32 variant of the same grid: plain FP32 sweeps (library depth) over a
    # fixed schedule that stays in FP32's stable range (levels 0..16, then 16
    # repeated); FP32 alone floors near kappa*eps32, so it is timed per sweep,
    # not to tolerance.
    f32 = None
    if not args.no_f32:
        levels = list(range(17)) + [16] * 20
        f32t = f.float()
        u32 = torch.zeros(npts, dtype=torch.float32, device="cuda")
        h32 = srj.srj_create(n, precision=srj.SRJ_PREC_F32, stream=stream.cuda_stream,
                             trace_capacity=64, temporal_depth=args.f32_depth)
        srj.srj_run_levels(h32, f32t.data_ptr(), u32.data_ptr(), levels)  # warm-up
        u32.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rn32 = srj.srj_run_levels(h32, f32t.data_ptr(), u32.data_ptr(), levels)
        e1.record(stream)
        torch.cuda.synchronize()
        srj.srj_destroy(h32)
        sw32 = sum(srj.srj_level_m(l) for l in levels)
        t32 = e0.elapsed_time(e1) * 1e-3
        d32 = args.f32_depth if args.f32_depth else 4
        passes32 = sum(srj.srj_level_m(l) // d32 + 1 for l in levels)
        pass32_s = t32 / passes32
        hbm_peak32, _ = peaks()
        f32 = {"glups": sw32 * npts / t32 / 1e9, "sweeps": sw32, "seconds": t32,
               "temporal_depth": d32,
               "hbm_per_pass_gbs": 12.0 * npts / pass32_s / 1e9,
               "hbm_per_pass_frac": 12.0 * npts / pass32_s / 1e9 / hbm_peak32,
               "effective_hbm_frac": 12.0 * sw32 * npts / t32 / 1e9 / hbm_peak32,
               "rel_residual_after": float(rn32[-1] / rn32[0]) if len(rn32) else None,
               "schedule": "levels 0..16 then 16 x20"}

    batched = None
    if not args.no_batched:
        batched = batched_leg(srj, inputs, torch, stream, seed=rank, fp64=not args.no_fp64)

    sel = None
    if not args.no_selector:
        sel = selector_leg(srj, inputs, torch, stream, seed=rank)
    mg = None
    if not args.no_mg:
        mg = mg_leg(srj, inputs, torch, stream, seed=rank)
        mg["srj_mixed_4096_time_to_tol_s"] = ms_max / args.steps / 1e3
    studies = None
    if not args.no_paper:
        studies = paper_studies_leg(srj, inputs, torch, stream, seed=rank)
    vark = None
    if not args.no_3d:
        vark = vark3d_leg(srj, inputs, torch, stream, seed=rank, side=args.side3d,
                          fp64=not args.no_fp64, depth=args.depth3d)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_line(float(os.environ.get("SRJ_ORACLE_SECONDS", "12")),
                                float(os.environ.get("SRJ_ORACLE_SECONDS_1CORE", "8")))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 sweeps on an FP32-pair iterate; f64 outer residual/update",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if side == SIDE else WORKLOAD.replace("4096x4096", "%dx%d" % (side, side)),
                       "grid": [side, side],
                       "precision": "mixed (FP64 refinement, FP32-pair inner)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (u+f FP64 268 MB, inner working set 335 MB)"},
            "time_to_tol_s": ms_max / args.steps / 1e3,
            "sweeps_per_solve": sweeps / args.steps, "outer_per_solve": outer / args.steps,
            "converged": ok, "rel_residual_check": rel_check,
            "roofline": {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak,
                         "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                         "traffic": profiled_traffic(),
                         "effective_achieved": hbm_effective,
                         "effective_frac": hbm_effective / hbm_peak,
                         "algorithmic_bytes_per_launch": algo_per_pass,
                         "bytes_moved_per_launch_by_design": moved_per_pass,
                         "sweeps_per_launch": sweeps_per_pass,
                         "launch_us": pass_s * 1e6,
                         "kernel": "wave2d_kernel<FP32-pair> inner pass; algorithmic 12 B per "
                                   "point per pass (read u, f; write u, FP32); effective_* "
                                   "counts the %.2f fused sweeps of a pass" % sweeps_per_pass,
                         "timing": "CUDA events around the inner cycle loops / passes",
                         "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, copy burst)"},
            "roofline_issue": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                               "unit": "T FP32-instr/s", "frac": alu_achieved / alu_peak,
                               "ops_per_update": DF_OPS_PER_LUP,
                               "peak_kind": "derived: 152 SMs x 128 FP32 lanes x median SM "
                                            "clock %.0f MHz" % sm_mhz},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * npts,
                    "d2h_bytes_per_step": 8 * npts},
            "gpu_launches": int(passes + 2 * outer + args.steps),
            "plain_fp64": fp64,
            "fp32_sweeps": f32,
            "batched": batched,
            "learned_selector": sel,
            "multigrid_srj_smoother": mg,
            "paper_studies": studies,
            "vark3d": vark,
            "mixed_vs_plain_speedup": (fp64["time_to_tol_s"] / (ms_max / args.steps / 1e3))
            if fp64 else None,
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f32", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-selector", action="store_true")
    ap.add_argument("--no-mg", action="store_true", help="skip the multigrid leg")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the Sec. 4.1 / Sec. 4.2.2 studies")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D variable-k leg")
    ap.add_argument("--with-3d", action="store_true", help=argparse.SUPPRESS)  # the default now
    ap.add_argument("--side3d", type=int, default=512)
    ap.add_argument("--depth3d", type=int, default=0,
                    help="sweeps per pass of the 3D mixed solve (0: library choice)")
    ap.add_argument("--f32-depth", type=int, default=0, help="temporal depth of the FP32 leg")
    ap.add_argument("--depth", type=int, default=0, help="temporal depth of the inner pass (0: library)")
    ap.add_argument("--side", type=int, default=SIDE, help="grid side (profiling runs only)")
    args = ap.parse_args()
    rank, world = (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    rank, world = dist_init()
    run_ours(args, rank, world)


if __name__ == "__main__":
    main()
