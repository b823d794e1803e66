#!/usr/bin/env python3
"""Throughput benchmark of the GB300 generalized-Stokes solver.

Metric: Stokes DOFs solved per second at true relative residual 1e-8, where
DOFs = 3 (2n+1)^3 + (n+1)^3 (velocity and pressure nodes including the
boundary, the paper's count for its throughput TPS). Workload: the 48^3-cube
Kuhn mesh of the unit cube with interior vertices jittered by up to 0.2 h
(seed 2), P2-P1, dt = 1e-3, mu in {1, 1e-2, 1e-4}, manufactured right-hand side,
Schur-complement CG with the Cahouet-Chabard preconditioner (C^Lambda).
One step = one solve for each of the three viscosities. Inputs are resident in
HBM; every matrix is larger than L2, so no separate L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (launched under torchrun) each rank solves its own replica of the
workload; value = all ranks' DOFs / the slowest rank's time ("replicas only":
the method has no data-parallel exchange step).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes DOFs solved per second at rel. residual 1e-8"
UNIT = "DOF/s"
N_DEFAULT = 48
MUS = (1.0, 1e-2, 1e-4)
DT = 1e-3
JITTER = 0.2
SEED = 2
TOL = 1e-8
CPU_SAMPLE_N = 8


def workload_name(n):
    return f"kuhn{n}^3-jitter0.2-P2P1-dt1e-3-mu{{1,1e-2,1e-4}}-schurCG-CLambda"


INNER_ITERS = 2
SCHUR_PREC, VEL_PREC = 0, 3
SCHUR_NAME = {0: "C^Lambda", 1: "C^Delta", 2: "C_lambda (B M_V^-1 B^T, 8 Chebyshev steps)"}
VEL_NAME = {3: "A~_3", 2: "A~_2 = A (3x3 blocks)", 1: "A~_1 = A + gamma mu D (3x3 blocks)"}


def config(n, precision):
    return {"workload": workload_name(n), "n_cubes": n, "mus": list(MUS), "dt": DT,
            "jitter": JITTER, "seed": SEED, "tol": TOL, "precision": precision,
            "dofs_per_solve": 3 * (2 * n + 1) ** 3 + (n + 1) ** 3,
            "solves_per_step": len(MUS), "method": "schur-cg", "schur_prec": SCHUR_NAME[SCHUR_PREC],
            "velocity_prec": VEL_NAME[VEL_PREC] + ", 1 V-cycle (Chebyshev-Jacobi degree 2)",
            "schur_inner": ("fixed %d PCG iterations on B Lambda^-1 B^T (1 V-cycle of M_Q + L_Q)" % INNER_ITERS
                            if INNER_ITERS > 0 else "PCG on B Lambda^-1 B^T to rel. 1e-1"),
            "coarse_levels": "replayed from captured CUDA graphs",
            "l2": "inputs larger than L2 (every matrix > 129 MB), no flush",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on bounded samples, on the host cores
# ---------------------------------------------------------------------------
CPU_TREND_N = (6, 8, 10, 12)


def oracle_step(n=CPU_SAMPLE_N, mus=MUS):
    """One oracle step on the n^3 sample: assembly + exact solve per viscosity."""
    import workload as wl
    from oracle.assemble import StokesSystem
    from oracle.mesh import KuhnMesh
    from oracle.solve import oracle_solve, relative_residual
    V = wl.kuhn_vertices(n, JITTER, SEED)
    t0 = time.perf_counter()
    worst = 0.0
    for mu in mus:
        s = StokesSystem(KuhnMesh(n, V), mu, DT)
        f = wl.manufactured_force(n, V, mu, DT, SEED)
        F = s.load(f)
        U, P = oracle_solve(s, F)
        worst = max(worst, relative_residual(s, U, P, F))
    return time.perf_counter() - t0, worst


def _oracle_task(arg):
    n, mus = arg
    t, w = oracle_step(n, mus)
    return n, len(mus), t, w


def oracle_on_all_cores(n, procs):
    """`procs` single-threaded oracle processes (spawned), each running one step
    of the n^3 sample (three viscosities); returns (aggregate DOF/s, wall s,
    worst residual)."""
    import multiprocessing as mp
    dofs = 3 * (2 * n + 1) ** 3 + (n + 1) ** 3
    with mp.get_context("spawn").Pool(procs) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_task, [(n, MUS)] * procs)
        wall = time.perf_counter() - t0
    return procs * len(MUS) * dofs / wall, wall, max(r[3] for r in res)


def oracle_trend(procs):
    """Single-thread oracle DOF/s per sample size (one viscosity, mu = 1e-2),
    the sizes solved concurrently, one process each."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(procs, len(CPU_TREND_N))) as pool:
        res = pool.map(_oracle_task, [(n, (1e-2,)) for n in CPU_TREND_N])
    return {str(n): (3 * (2 * n + 1) ** 3 + (n + 1) ** 3) * k / t for n, k, t, _ in res}


def cpu_baseline_worker(steps):
    """Runs in a child process with single-threaded BLAS and no GPU."""
    procs = os.cpu_count() or 1
    trend = oracle_trend(procs)
    vals, walls, worst = [], [], 0.0
    for _ in range(steps):
        v, w, r = oracle_on_all_cores(CPU_SAMPLE_N, procs)
        vals.append(v)
        walls.append(w)
        worst = max(worst, r)
    print(json.dumps({"value": statistics.median(vals), "wall_s": statistics.median(walls), "procs": procs,
                      "trend": trend, "worst_residual": worst, "steps": steps}))


def cpu_sample_text(procs, wall=None):
    w = f", {wall:.1f} s wall per step" if wall else ""
    return (f"oracle (COO assembly + exact Schur CG with sparse-LU inner solves) on the {CPU_SAMPLE_N}^3 jittered "
            f"sample of this workload, mu in {{1,1e-2,1e-4}}, dt=1e-3: {procs} single-threaded processes "
            f"(one per host core) each solving the three viscosities{w}")


def run_cpu_baseline(steps=1):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker",
                          str(steps)], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "error": out.stderr[-300:]}
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": r["value"], "unit": UNIT, "cores": r["procs"], "kind": "oracle",
            "sample": cpu_sample_text(r["procs"], r["wall_s"]),
            "threads_per_process": 1,
            "per_core_trend_dofs_per_s": r["trend"],
            "per_core_trend_sample": "one oracle process per size, mu = 1e-2, sizes n^3 run concurrently",
            "worst_residual": r["worst_residual"]}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.dev = device_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.send_signal(signal.SIGTERM)
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [x for x in sm if x >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha():
    """Hash of the files that define the sparse kernels (sparse.cu, sym3.cu, internal.h)."""
    h = hashlib.sha256()
    for name in ("sparse.cu", "sym3.cu", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2407_01783_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name):
    """Per-launch DRAM bytes of `kernel_name` from a committed ncu summary, if the
    summary was taken on the current kernel source."""
    sha = kernel_source_sha()
    prof = os.path.join(ROOT, "profiles")
    if not os.path.isdir(prof):
        return None
    for fn in sorted(os.listdir(prof)):
        if not fn.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(prof, fn)):
            m = re.search(r"bench-traffic: kernel=(\w+) bytes_per_launch=([0-9.eE+]+) sparse_cu_sha=(\w+)", line)
            if m and m.group(1) == kernel_name and m.group(3) == sha:
                return float(m.group(2))
    return None


# ---------------------------------------------------------------------------
# multi-rank helpers (replicas only: the ranks exchange nothing but timings)
# ---------------------------------------------------------------------------
def event_overhead_ms(torch, dev, trials=64):
    """Time that a pair of CUDA events adds around one launch: the median
    elapsed time of events bracketing an empty (zero-cycle) kernel. The warm-up
    per-class times (events around every launch) have it subtracted once per
    launch before the classes are ranked, so that small, frequent kernels are
    not over-weighted against the device times of an ncu launch list."""
    stream = torch.cuda.current_stream(dev)
    ts = []
    for _ in range(trials):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda._sleep(0)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def max_over_ranks(x, dist, device):
    """Largest value of x over all ranks (x itself when not distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, solves_per_step, dofs, ms_per_step):
    """Whole-job throughput: every rank solves its own replica of the workload."""
    return world * solves_per_step * dofs / (ms_per_step / 1e3)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import workload as wl
    import paper_2407_01783_gb300 as sk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.only_lockstep:
        return run_lockstep(sk, torch, wl, dev, world, dist, n=args.lockstep_n)

    n = args.n
    V = wl.kuhn_vertices(n, JITTER, SEED)
    dofs = 3 * (2 * n + 1) ** 3 + (n + 1) ** 3
    prec = sk.PRECISION_MIXED if args.precision == "mixed" else sk.PRECISION_FP64

    mus = tuple(args.mus) if args.mus else MUS

    setup_times = []

    def make(precision, profile, **extra):
        solvers, fs, outs = [], [], []
        for mu in mus:
            opt = sk.stokes_default_options(precision=precision, profile=profile, vcycles=args.vcycles,
                                            schur_inner_iters=args.schur_inner_iters, format=args.format,
                                            vel_prec=args.vel_prec, schur_prec=args.schur_prec,
                                            **({"inner_tol": args.inner_tol} if args.inner_tol else {}),
                                            **({"pass_tol": args.pass_tol} if args.pass_tol else {}),
                                            **extra)
            torch.cuda.synchronize()
            t_s = time.perf_counter()
            S = sk.Stokes(n, V, mu, DT, 0.0, opt, device=dev)
            torch.cuda.synchronize()
            setup_times.append(time.perf_counter() - t_s)
            f = torch.as_tensor(wl.manufactured_force(n, V, mu, DT, SEED), device=dev)
            u = torch.empty_like(f)
            p = torch.empty(S.n_p1, dtype=torch.float64, device=dev)
            solvers.append(S)
            fs.append(f)
            outs.append((u, p))
        return solvers, fs, outs

    def step(solvers, fs, outs, infos):
        for S, f, (u, p) in zip(solvers, fs, outs):
            _, _, info = S.solve(f, None, TOL, out=(u, p))
            infos.append(info.as_dict())

    def class_stats(solvers):
        out = {}
        for name, kid in sk.KERNEL.items():
            cnt, kms, kbytes = 0, 0.0, 0.0
            for S in solvers:
                c_, m_, b_ = sk.stokes_kernel_stats(S.ctx, kid)
                cnt += c_
                kms += m_
                kbytes += b_
            out[name] = {"launches": cnt, "ms": kms, "bytes": kbytes}
        return out

    warm_stats = {}
    warm_stats_meta = {}

    def timed(solvers, fs, outs, steps, warmup, clocks=None):
        infos = []
        for _ in range(warmup):
            step(solvers, fs, outs, infos)
        if solvers[0].options.profile:
            # warm-up steps time every kernel class; the timed steps put CUDA
            # events only around the dominant class (all launches are counted)
            warm_stats.update(class_stats(solvers))
            eps_ms = event_overhead_ms(torch, dev)
            for v in warm_stats.values():
                v["device_ms"] = max(0.0, v["ms"] - v["launches"] * eps_ms)
            warm_stats_meta["event_overhead_us"] = 1e3 * eps_ms
            dom_w = max(warm_stats, key=lambda k: warm_stats[k]["device_ms"])
            for S in solvers:
                sk.stokes_profile_mode(S.ctx, 2 + sk.KERNEL[dom_w])
        for S in solvers:
            sk.stokes_kernel_stats_reset(S.ctx)
        infos = []
        stream = torch.cuda.current_stream(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        if clocks:
            clocks.start()
        e0.record(stream)
        for _ in range(steps):
            step(solvers, fs, outs, infos)
        e1.record(stream)
        barrier()
        ck = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, dev)
        return ms, infos, ck

    solvers, fs, outs = make(prec, 1)
    torch.cuda.synchronize()
    # stokes_setup alone (the first context also tunes the threads per row,
    # cached for the others); host-side input generation is not included
    setup_s = statistics.mean(setup_times)
    setup_phases = [sk.stokes_setup_phases(S.ctx) for S in solvers]
    clocks = Clocks(local)
    ms, infos, ck = timed(solvers, fs, outs, args.steps, args.warmup, clocks)
    worst = max(i["rel_residual"] for i in infos)
    bad = [i for i in infos if i["status"] != 0]
    value = job_value(world, len(mus), dofs, ms)

    # per-kernel statistics: launches of every class and CUDA-event times of the
    # dominant class over the timed region; shares from the warm-up steps
    kinfo = class_stats(solvers)
    peak, peak_kind = measured_peak_gbs()
    total_launches = sum(v["launches"] for v in kinfo.values())
    dom = max(warm_stats, key=lambda k: warm_stats[k]["device_ms"])
    # the dominant class's launches that ran outside graph replays were timed
    # with CUDA events on the solver's stream over the timed region
    tl, tms, tby = 0, 0.0, 0.0
    for S in solvers:
        a_, b_, c_ = sk.stokes_kernel_timing(S.ctx, sk.KERNEL[dom])
        tl, tms, tby = tl + a_, tms + b_, tby + c_
    d = {"launches": tl, "ms": tms, "bytes": tby}
    achieved = (d["bytes"] / d["launches"]) / (d["ms"] / d["launches"] / 1e3) / 1e9 if d["launches"] else 0.0
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": ncu_traffic(dom),
                "bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
                "timed_launches": d["launches"],
                "launches_in_timed_region": kinfo[dom]["launches"]}
    wtot = max(1e-12, sum(x["device_ms"] for x in warm_stats.values()))
    kernels = {}
    for k, v in warm_stats.items():
        gbs = (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None
        kernels[k] = {"launches_per_step": kinfo[k]["launches"] / args.steps,
                      "share_warmup": v["device_ms"] / wtot,
                      "GBps_warmup": gbs,
                      "frac_warmup": (gbs / peak) if gbs else None,
                      "device_ms_per_step_warmup": v["device_ms"] / max(1, args.warmup),
                      "avg_launch_us_warmup": 1e3 * v["ms"] / max(1, v["launches"])}

    # end to end through the public API with HOST buffers (copies inside the timing)
    fh = [torch.empty_like(f, device="cpu").pin_memory() for f in fs]
    for a, b in zip(fh, fs):
        a.copy_(b)
    fh_np = [a.numpy() for a in fh]
    uh = [torch.empty_like(f, device="cpu").pin_memory().numpy() for f in fs]
    ph = [torch.empty(S.n_p1, dtype=torch.float64).pin_memory().numpy() for S in solvers]
    e2e_ms = []
    for it in range(0 if args.no_e2e else args.warmup + args.steps):
        barrier()
        t0 = time.perf_counter()
        for S, f, u, p in zip(solvers, fh_np, uh, ph):
            sk.stokes_solve_host(S.ctx, f, None, TOL, u, p)
        barrier()
        if it >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_step = max_over_ranks(statistics.mean(e2e_ms) if e2e_ms else float("nan"), dist, dev)
    h2d = sum(a.nbytes for a in fh_np)
    d2h = sum(a.nbytes for a in uh) + sum(a.nbytes for a in ph)
    for S in solvers:
        S.close()
    del solvers

    fp64 = fp64_sched = mixed_err = None
    if prec == sk.PRECISION_MIXED and not args.no_fp64:
        def fp64_line(sched, label):
            s2, f2, o2 = make(sk.PRECISION_FP64, 0, pass_schedule=sched)
            ms64, inf64, _ = timed(s2, f2, o2, max(1, args.steps // 2), max(1, args.warmup // 2))
            line_ = {"value": job_value(world, len(mus), dofs, ms64), "ms_per_step": ms64, "schedule": label,
                     "worst_residual": max(i["rel_residual"] for i in inf64),
                     "iters": [(i["outer_iters"], i["inner_iters"], i["refinements"]) for i in inf64[:len(mus)]]}
            return line_, s2, f2, o2
        fp64, s2, _, _ = fp64_line(2, "one pass aimed at 1e-8, inner velocity solves to 1e-10 (the paper's setting)")
        for S in s2:
            S.close()
        fp64_sched, s2, f2, o2 = fp64_line(1, "the mixed line's schedule: passes asking for a 3e-2 reduction, "
                                              "inner velocity solves to 1e-3")
        # error of the mixed-precision solutions (1e-8) against FP64 solves of the
        # same systems to 1e-12
        mixed_err = []
        for S, f, (u64, p64), (um, pm) in zip(s2, f2, o2, outs):
            S.solve(f, None, 1e-12, out=(u64, p64))
            mixed_err.append({"mu": S.mu,
                              "velocity_rel_l2": float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64)),
                              "pressure_rel_l2": float(torch.linalg.norm(pm - p64) / torch.linalg.norm(p64))})
        for S in s2:
            S.close()

    coupled = None
    if not args.no_coupled:
        s3, f3, o3 = make(prec, 0, method=sk.METHOD_COUPLED, block_lu=1)
        ms2, inf2, _ = timed(s3, f3, o3, max(1, args.steps // 2), max(1, args.warmup // 2))
        coupled = {"value": job_value(world, len(mus), dofs, ms2), "ms_per_step": ms2,
                   "method": "coupled FGMRES(30), block-LU preconditioner, V-cycles for A~^{-1}",
                   "worst_residual": max(i["rel_residual"] for i in inf2),
                   "iters": [(i["outer_iters"], i["refinements"]) for i in inf2[:len(mus)]]}
        for S in s3:
            S.close()

    lockstep = None
    if not args.no_batched:
        lockstep = run_lockstep(sk, torch, wl, dev, world, dist, n=args.lockstep_n)

    concurrent = None
    if not args.no_concurrent:
        concurrent = run_concurrent(sk, torch, wl, dev, world, dist, n, V, mus, prec, args)

    batched = None
    if not args.no_batched:
        batched = run_batched(sk, torch, wl, dev, world, dist)

    coupled96 = None
    if not args.no_coupled96:
        coupled96 = run_coupled96(sk, torch, wl, dev, world, dist)

    if rank != 0:
        return None
    cpu = run_cpu_baseline(1) if (world == 1 and not args.no_cpu) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == sk.PRECISION_MIXED else "f64",
        "data": "synthetic (seeded jittered Kuhn mesh, manufactured solution)",
        "config": config(n, args.precision) if not args.mus else dict(config(n, args.precision), mus=list(mus)),
        "clocks": ck,
        "e2e": {"value": job_value(world, len(mus), dofs, e2e_step), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step},
        "gpu_launches": int(total_launches),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "setup_s_per_instance": setup_s,
        "setup_s_each": setup_times[:len(mus)],
        "setup_phases_ms": setup_phases,
        "worst_rel_residual": worst,
        "failed_solves": len(bad),
        "iters": [(i["outer_iters"], i["inner_iters"], i["refinements"]) for i in infos[:3]],
        "kernels": kernels,
        "kernels_note": ("shares: warm-up solves with CUDA events around every launch (no graphs), minus the "
                         "measured event overhead per launch (%.2f us)" % warm_stats_meta.get("event_overhead_us", 0.0)),
        "plain_fp64": fp64,
        "plain_fp64_same_schedule": fp64_sched,
        "mixed_error_vs_fp64_1e-12": mixed_err,
        "method2_coupled": coupled,
        "concurrent_viscosities": concurrent,
        "lockstep_rhs": lockstep,
        "batched": batched,
        "coupled_96": coupled96,
    }
    return line


def run_lockstep(sk, torch, wl, dev, world, dist, n=40, rhs=4, reps=3, mu=1e-2, dt=1e-3):
    """One instance of the batch's kind (n^3 jittered Kuhn mesh, mu = 1e-2,
    dt = 1e-3, mixed precision, coupled FGMRES + block-LU, one V-cycle) with
    `rhs` N(0,1) forces: one stokes_solve_multi call (the forces in lockstep)
    against the forces solved one after another. One warm-up, then `reps`
    timed calls each (CUDA events)."""
    V = wl.kuhn_vertices(n, JITTER, 7)
    opt = sk.stokes_default_options(precision=sk.PRECISION_MIXED, vcycles=1, method=sk.METHOD_COUPLED)
    S = sk.Stokes(n, V, mu, dt, 0.0, opt, device=dev)
    F = torch.stack([torch.as_tensor(wl.random_force(n, 50 + k), device=dev).reshape(S.n_p2, 3)
                     for k in range(rhs)]).contiguous()
    U = torch.empty_like(F)
    P = torch.empty(rhs, S.n_p1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed_call(fn):
        fn()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts), out

    ms_multi, infos = timed_call(lambda: S.solve_multi(F, None, TOL, out=(U, P))[2])
    ms_one, infos1 = timed_call(lambda: [S.solve(F[k], None, TOL, out=(U[k], P[k]))[2] for k in range(rhs)])
    S.close()
    dofs = (3 * (2 * n + 1) ** 3 + (n + 1) ** 3) * rhs
    ms_multi = max_over_ranks(ms_multi, dist, dev)
    ms_one = max_over_ranks(ms_one, dist, dev)
    return {"workload": f"kuhn{n}^3-jitter0.2-P2P1-mu{mu:g}-dt{dt:g}-coupledFGMRES-{rhs}xN(0,1)", "rhs": rhs,
            "value": world * dofs / (ms_multi / 1e3), "unit": UNIT, "ms": ms_multi,
            "one_at_a_time": {"value": world * dofs / (ms_one / 1e3), "ms": ms_one},
            "outer_iters": [i.outer_iters for i in infos], "outer_iters_one_at_a_time": [i.outer_iters for i in infos1],
            "worst_residual": max(i.rel_residual for i in infos)}


def run_concurrent(sk, torch, wl, dev, world, dist, n, V, mus, prec, args, reps=3):
    """The main line's solves (same mesh, loads, options and tolerance) with
    the viscosities as concurrent instances: one context, CUDA stream and host
    thread each (StokesBatch), so one solve's latency-bound stretches (coarse
    levels, small vector kernels, host reads) overlap another's bandwidth-bound
    sweeps. One warm-up step, then `reps` steps timed with CUDA events."""
    spec = [(n, V, mu, DT, 0.0) for mu in mus]
    opt = sk.stokes_default_options(precision=prec, vcycles=args.vcycles, schur_inner_iters=args.schur_inner_iters,
                                    format=args.format, vel_prec=args.vel_prec, schur_prec=args.schur_prec)
    B = sk.StokesBatch(spec, opt, device=dev, host_wait=0)
    forces = [torch.as_tensor(wl.manufactured_force(n, V, mu, DT, SEED), device=dev).reshape(1, -1, 3) for mu in mus]
    outs, _, _ = B.solve_all(forces, TOL)
    times, flat = [], []
    for _ in range(reps):
        _, infos, ms_ = B.solve_all(forces, TOL, outs)
        times.append(ms_)
        flat += [x for inf in infos for x in inf]
    B.close()
    ms = max_over_ranks(statistics.mean(times), dist, dev)
    dofs = 3 * (2 * n + 1) ** 3 + (n + 1) ** 3
    return {"value": job_value(world, len(mus), dofs, ms), "unit": UNIT, "ms_per_step": ms, "steps": reps,
            "worst_residual": max(x["rel_residual"] for x in flat),
            "failed": sum(1 for x in flat if x["status"] != 0),
            "scheme": "the %d viscosities of one step as concurrent instances (one context + stream + host "
                      "thread each); the main value solves them one after another" % len(mus)}


def run_batched(sk, torch, wl, dev, world, dist, count=32, rhs=4):
    """Uneven batch: `count` seeded instances (n in 12..40, mu log-U[1e-4, 1],
    dt log-U[1e-4, 1e-2]), `rhs` N(0,1) body forces each, solved concurrently
    (one stream per instance), mixed precision, to the same tolerance, with
    the coupled FGMRES form (no inner Krylov solves, so few host
    synchronisations). Each instance's right-hand sides go through one
    stokes_solve_multi call (four systems in lockstep sharing every V-cycle,
    mass-inverse and vector-kernel sweep); the same batch with the right-hand
    sides solved one after another is timed beside it."""
    insts = wl.batched_instances(count, seed=4)
    spec = [(i.n, i.vertices(), i.mu, i.dt, 0.0) for i in insts]
    B = sk.StokesBatch(spec, sk.stokes_default_options(precision=sk.PRECISION_MIXED, vcycles=1,
                                                       method=sk.METHOD_COUPLED), device=dev)
    forces = B.stack([[torch.as_tensor(wl.random_force(i.n, i.seed * 10 + k), device=dev) for k in range(rhs)]
                      for i in insts])
    dofs = sum(B.dofs) * rhs
    timings = {}
    for multi in (False, True):
        B.multi = multi
        outs, _, _ = B.solve_all(forces, TOL)                 # warm-up (workspace, graphs)
        _, infos, ms = B.solve_all(forces, TOL, outs)
        timings[multi] = (max_over_ranks(ms, dist, dev), infos)
    B.close()
    ms, infos = timings[True]
    ms1, infos1 = timings[False]
    flat = [x for inf in infos for x in inf]
    flat1 = [x for inf in infos1 for x in inf]
    return {"value": world * dofs / (ms / 1e3), "unit": UNIT, "ms_per_batch": ms,
            "instances": count, "rhs_per_instance": rhs, "dofs_per_batch": dofs,
            "n_range": [min(i.n for i in insts), max(i.n for i in insts)],
            "worst_residual": max(x["rel_residual"] for x in flat),
            "failed": sum(1 for x in flat if x["status"] != 0),
            "one_rhs_at_a_time": {"value": world * dofs / (ms1 / 1e3), "ms_per_batch": ms1,
                                  "worst_residual": max(x["rel_residual"] for x in flat1),
                                  "failed": sum(1 for x in flat1 if x["status"] != 0)},
            "scheme": "one context + stream per instance, host thread per instance, mixed precision, "
                      "coupled FGMRES(30) + block-LU, the 4 right-hand sides of an instance in lockstep "
                      "(stokes_solve_multi), V-cycles and C replayed from CUDA graphs"}


def run_coupled96(sk, torch, wl, dev, world, dist, n=96, mu=1e-3, dt=1e-3, gammas=(0.0, 1.0, 10.0), seed=3):
    """Fully coupled form on the 96^3 jittered mesh: block-triangular FGMRES(30)
    vs the Schur form, mixed precision, for each augmented-Lagrangian gamma.
    One untimed solve, then one solve timed with CUDA events, per case."""
    V = wl.kuhn_vertices(n, JITTER, seed)
    f = torch.as_tensor(wl.manufactured_force(n, V, mu, dt, seed), device=dev)
    dofs = 3 * (2 * n + 1) ** 3 + (n + 1) ** 3
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"kuhn{n}^3-jitter0.2-P2P1-dt1e-3-mu1e-3-gamma{{0,1,10}}", "seed": seed, "mu": mu, "dt": dt,
           "dofs": dofs, "cases": []}
    for gamma in gammas:
        for label, extra in (("fgmres_block_triangular", dict(method=sk.METHOD_COUPLED, block_lu=0)),
                             ("schur_cg", dict(method=sk.METHOD_SCHUR))):
            opt = sk.stokes_default_options(precision=sk.PRECISION_MIXED, vcycles=1, **extra)
            S = sk.Stokes(n, V, mu, dt, gamma, opt, device=dev)
            u = torch.empty_like(f)
            p = torch.empty(S.n_p1, dtype=torch.float64, device=dev)
            S.solve(f, None, TOL, out=(u, p))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, info = S.solve(f, None, TOL, out=(u, p))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
            S.close()
            out["cases"].append({"gamma": gamma, "method": label, "ms": ms,
                                 "value": world * dofs / (ms / 1e3), "unit": UNIT,
                                 "outer_iters": info.outer_iters, "inner_iters": info.inner_iters,
                                 "refinements": info.refinements, "rel_residual": info.rel_residual,
                                 "status": info.status})
    return out


def run_reference(args):
    """The oracle as it stands on the host cores: every step runs one
    single-threaded oracle process per core, each solving the three
    viscosities of the 8^3 sample of the workload (spawned processes, BLAS
    threads set to 1 before they start)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return None
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    procs = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_on_all_cores(CPU_SAMPLE_N, procs)
    vals, walls, worst = [], [], 0.0
    for _ in range(args.steps):
        v, w, r = oracle_on_all_cores(CPU_SAMPLE_N, procs)
        vals.append(v)
        walls.append(w)
        worst = max(worst, r)
    value = statistics.mean(vals)
    sec = statistics.mean(walls)
    cfg = dict(config(args.n, "fp64"), workload=f"{workload_name(args.n)} (oracle on the {CPU_SAMPLE_N}^3 sample)",
               sample_n_cubes=CPU_SAMPLE_N)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded jittered Kuhn mesh, manufactured solution)",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": cpu_sample_text(procs, sec), "threads_per_process": 1},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "worst_rel_residual": worst}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-coupled", action="store_true", help="skip the Method 2 (coupled FGMRES) line")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven-batch line")
    ap.add_argument("--no-concurrent", action="store_true",
                    help="skip the line with the step's viscosities solved concurrently")
    ap.add_argument("--lockstep-n", type=int, default=40, help="mesh size of the lockstep right-hand-side line")
    ap.add_argument("--only-lockstep", action="store_true",
                    help="run only the lockstep right-hand-side line (profiling) and print it")
    ap.add_argument("--no-coupled96", action="store_true", help="skip the 96^3 coupled-vs-Schur comparison")
    ap.add_argument("--mus", type=float, nargs="*", default=None, help="viscosities (default 1 1e-2 1e-4)")
    ap.add_argument("--vcycles", type=int, default=1, help="V-cycles per A~_3 preconditioner application")
    ap.add_argument("--inner-tol", type=float, default=None, help="override options.inner_tol")
    ap.add_argument("--pass-tol", type=float, default=None, help="override options.pass_tol")
    ap.add_argument("--schur-prec", type=int, default=0, choices=[0, 1, 2],
                    help="Schur preconditioner C^Lambda (default), C^Delta or C_lambda (M_V)")
    ap.add_argument("--vel-prec", type=int, default=3, choices=[1, 2, 3],
                    help="velocity preconditioner A~_1, A~_2 or A~_3 (default)")
    ap.add_argument("--format", type=int, default=0,
                    help="matrix storage: 0 stencil on large levels, 1 CSR, 2 stencil everywhere")
    ap.add_argument("--schur-inner-iters", type=int, default=2,
                    help="fixed PCG iterations inside C (0: stop at the inner tolerance)")
    ap.add_argument("--cpu-baseline-worker", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_baseline_worker:
        cpu_baseline_worker(args.cpu_baseline_worker)
        return
    if args.warmup < 3:
        args.warmup = 3
    global INNER_ITERS, SCHUR_PREC, VEL_PREC
    INNER_ITERS = args.schur_inner_iters
    SCHUR_PREC, VEL_PREC = args.schur_prec, args.vel_prec
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
