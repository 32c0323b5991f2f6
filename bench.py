#!/usr/bin/env python
"""Benchmark of the multiscale multibasis pressure solver on one GB300.

Metric: fine-cell unknowns per second to a 1e-6 relative residual, for one
pass of the whole hot path per step on the 3D 60x220x85 geomodel
(1,122,000 cells; top 35 layers lognormal with Kz = 0.1 Kx, bottom 50 layers
1000:1 binary channels; 6x11x17 coarse blocks of 10x20x5):

    TPFA assembly -> MsRSB basis smoothing from the block indicator to
    increment 1e-3 -> Galerkin A_c = P^T A P -> dense coarse factor/inverse ->
    multiscale + ILU(0) solve from p = 0 to ||q - A p|| <= 1e-6 ||q||, with
    GMRES(30) right-preconditioned by the multistage cycle (Sec. 5.2 gives
    Richardson or GMRES as the outer iteration); Richardson is timed beside it

Inputs (permeability, sources) are resident in HBM when the timed region
starts; the integer analysis (connection list, wavefront levels, support
patterns) is done once per grid before timing.  The headline is the plain
FP64 form; the mixed form (FP32 basis / smoother / coarse inverse, FP64 outer
residual and refinement) is reported beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own seeded geomodel (replicas; weak scaling).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

from paper_2001_01624_gb300 import replicas as R

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("3D 60x220x85 Cartesian (1,122,000 cells), TPFA 7-point, top 35 layers lognormal "
            "(ln K ~ N(ln 100 mD, 2^2), corr 8 cells, Kz=0.1Kx), bottom 50 layers binary channels 1000:1 "
            "(Kz=0.1Kx); 6x11x17 coarse blocks of 10x20x5; MsRSB omega 2/3 to 1e-3; MS+ILU(0) cycle as "
            "preconditioner of GMRES(30) to 1e-6")
OUTER = {"gmres": (1, 30), "richardson": (0, 30)}
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 rate of the GB300
METRIC = "fine-cell unknowns/sec to 1e-6 rel residual (full hot path per step)"
UNIT = "unknowns/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-single", action="store_true",
                    help="also time one full step of the single-threaded oracle (about a minute)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-fv", action="store_true")
    ap.add_argument("--no-cpr", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the faulted c3 solves, the ensemble and the serving summaries of the default line")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run N extra untimed steps only (for ncu launch lists)")
    ap.add_argument("--profile-mixed", action="store_true",
                    help="with --profile-steps: the mixed-precision plan only")
    ap.add_argument("--profile-ilu", type=int, default=0,
                    help="only assemble the c2 system and apply ILU(0) N times in each precision (for ncu captures)")
    ap.add_argument("--nz", type=int, default=85, help="--profile-ilu: layers of the 60x220 grid")
    ap.add_argument("--faulted", action="store_true",
                    help="--profile-ilu: the faulted 200x200x50 geomodel instead (segment sweeps)")
    ap.add_argument("--profile-coarse-sweep", action="store_true",
                    help="only form the FP64 and mixed Galerkin coarse operators of the 60x220x85 geomodel (their "
                         "sweep inverses; for ncu captures)")
    ap.add_argument("--profile-coarse", action="store_true",
                    help="only form the finite-volume coarse operator of the 60x220x85 geomodel (Gauss-Jordan "
                         "inverse; for ncu captures)")
    ap.add_argument("--workload", choices=["c2", "ensemble", "serving", "coupling"], default="c2",
                    help="c2: the 60x220x85 geomodel (headline); ensemble: the batched uneven ensemble; "
                         "serving: Poisson stream of two-phase time steps on resident geomodels; coupling: "
                         "viscosity-ratio study of dynamic bases on a 42x22 field")
    ap.add_argument("--models", type=int, default=32, help="serving: resident geomodels")
    ap.add_argument("--requests", type=int, default=400, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrival rate (requests/s)")
    ap.add_argument("--members", type=int, default=256, help="ensemble members")
    ap.add_argument("--workers", type=int, default=16, help="ensemble worker streams")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from profiles/ncu_traffic.txt, or None
    when absent or when the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        f = ln.split()
        if len(f) >= 4 and len(f) % 2 == 0 and f[0] == kernel:
            # then one or more (source file, sha256[:16] at capture) pairs
            for name, sha in zip(f[2::2], f[3::2]):
                src = os.path.join(ROOT, "paper_2001_01624_gb300", "csrc", name)
                if not os.path.exists(src):
                    return None
                if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != sha:
                    return None
            return float(f[1])
    return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# ---------------------------------------------------------------- oracle leg
def host_cpu():
    """(logical CPUs, CPU model) of this host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":", 1)
                if len(k) == 2 and k[0].strip() in ("model name", "Model name"):
                    model = k[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.startswith("Model name:"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_full_step(gm, openmp=True, outer="gmres"):
    """One complete step of the workload by the CPU oracle, nothing sampled or
    extrapolated: assembly, pin, partition, supports, MsRSB basis to increment
    1e-3, Galerkin, Cholesky, ILU(0) factors, and the solve from p = 0 to
    1e-6.  openmp selects the OpenMP build (all host cores) or the
    single-threaded correctness build.  Returns dict(seconds, phases, counts,
    threads)."""
    import oracle as O
    O.use_openmp(openmp)
    try:
        threads = O.openmp_threads() if openmp else 1
        ph = {}
        t0 = time.perf_counter()
        s = O.assemble_tpfa(gm.grid, gm.perm)
        Ap, qp = O.pin(s.A, gm.q_active(), 0)
        part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
        sp, sc = O.support_box(gm.grid, s.cells, s.A, part, M, gm.block)
        t1 = time.perf_counter()
        B = O.msrsb_basis(s.A, part, M, sp, sc, 2.0 / 3.0, 1e-3, 500)
        t2 = time.perf_counter()
        L = O.cholesky(O.galerkin(Ap, B))
        lu = O.ilu0(Ap)
        t3 = time.perf_counter()
        if outer == "gmres":
            r = O.ms_gmres(Ap, [(B, L)], qp, tol=1e-6, max_iter=5000, restart=OUTER["gmres"][1], lu=lu)
        else:
            r = O.ms_solve(Ap, [(B, L)], qp, tol=1e-6, max_iter=5000, lu=lu)
        t4 = time.perf_counter()
    finally:
        O.use_openmp(False)
    ph = {"setup": t1 - t0, "basis": t2 - t1, "coarse_ilu": t3 - t2, "solve": t4 - t3}
    return {"seconds": t4 - t0, "phases": {k: round(v, 3) for k, v in ph.items()}, "basis_iters": int(B.iters),
            "steps": int(r.iters), "converged": bool(r.converged), "threads": threads}


def cpu_baseline_line(n, res, what="one full step of the same workload"):
    nproc, model = host_cpu()
    build = (f"OpenMP build on {res['threads']} threads" if res["threads"] > 1
             else "single-threaded build")
    return {"value": n / res["seconds"], "unit": UNIT, "cores": res["threads"], "kind": "oracle",
            "sample": f"{what} (basis {res['basis_iters']} iterations, GMRES(30) {res['steps']} steps) by the "
                      f"oracle (plain C, FP64), {build}; timed in full, nothing extrapolated",
            "seconds": res["seconds"], "phases": res["phases"], "nproc": nproc, "cpu_model": model}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2001_01624_gb300 import geomodel as G
    import oracle as O
    O.build()
    O.build(openmp=True)
    gm = G.config2(0)
    n = gm.grid.n_active()
    for _ in range(args.warmup):
        oracle_full_step(gm)
    runs = [oracle_full_step(gm) for _ in range(args.steps)]
    tot = sum(r["seconds"] for r in runs)
    v = n * len(runs) / tot
    cb = cpu_baseline_line(n, runs[-1], what=f"{len(runs)} full steps of the same workload, each")
    cb["value"] = v
    cb["seconds"] = tot / len(runs)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(runs), "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(runs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": n, "precision": "fp64", "parallelism": "replicas"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU leg
class Plan:
    """Handles for one geomodel and one precision: analysis done once."""

    def __init__(self, ms, ctx, gm, prec, dev, torch):
        self.ms, self.ctx, self.prec = ms, ctx, prec
        self.sys = ms.ms_system_create(ctx, gm.grid, 0)
        self.perm = torch.from_numpy(gm.perm.ravel().copy()).to(dev)
        self.q = torch.from_numpy(gm.q_active()).to(dev)
        self.p = torch.zeros_like(self.q)
        ms.ms_assemble_tpfa(ctx, self.sys, self.perm)
        part, M = ms.ms_partition_cartesian(ctx, self.sys, gm.block)
        self.basis, _ = ms.ms_build_basis(ctx, self.sys, part, M, block=gm.block, precision=prec)
        self.coarse = ms.ms_galerkin(ctx, self.sys, self.basis, prec)
        self.n = ms.ms_system_get_info(self.sys)["n"]
        self.M = M

    def step(self, perm=None, q=None, p=None, outer="gmres", coarse=None):
        ms, ctx = self.ms, self.ctx
        coarse = self.coarse if coarse is None else coarse
        ms.ms_assemble_tpfa(ctx, self.sys, self.perm if perm is None else perm)
        bit = ms.ms_basis_rebuild(ctx, self.sys, self.basis)
        ms.ms_coarse_refresh(ctx, self.sys, coarse)
        o, m = OUTER[outer]
        info = ms.ms_solve(ctx, self.sys, [coarse], self.q if q is None else q, self.p if p is None else p,
                           tol=1e-6, max_iter=5000, precision=self.prec, outer=o, restart=m)
        info["basis_iters"] = bit
        return info

    def release(self):
        self.ms.ms_coarse_release(self.coarse)
        self.ms.ms_basis_release(self.basis)
        self.ms.ms_system_release(self.sys)


def timed_steps(torch, plan, stream, K, dist, world, outer="gmres", coarse=None):
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [plan.step(outer=outer, coarse=coarse) for _ in range(K)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms_tot = e0.elapsed_time(e1)
    if world > 1:
        ms_tot = R.max_over_ranks(dist, [ms_tot], "cuda")[0]
        dist.barrier()
    return ms_tot, infos


ENSEMBLE = ("batched ensemble of {m} independent 3D TPFA systems of uneven size (nx, ny ~ U{{24..96}}, "
            "nz ~ U{{8..48}}, 20k <= N <= 400k; lognormal K, correlation U[2,16] cells, sigma U[1,3], standard "
            "field clipped to +-3, Kz = 0.1 Kx; seed 1000+m); 8x8x4 coarse blocks; per step every member's MsRSB "
            "basis re-smoothed (all members in one persistent launch), Galerkin "
            "operator re-formed and GMRES(30) with the MS+ILU(0) cycle as preconditioner to 1e-6, FP32 bulk / FP64 "
            "residual")


def c3_extra(torch, ms, G, dev, stream):
    """The faulted 200x200x50 geomodel (config 3): general + static stages,
    GMRES(30) to 1e-6 in FP64 and mixed, and Richardson with the Dp(Inf)
    dynamic stage (mixed); wall times of the basis setup and device-timed
    solves."""
    import numpy as np
    gm = G.config3(0)
    ctx = ms.ms_create(dev.index or 0, stream)
    out = {"workload": "faulted 200x200x50 (1,840,020 active cells, 6 faults with 2-cell throw), general 10x10x5 "
                       "+ facies static stage"}
    try:
        t0 = time.perf_counter()
        s = ms.ms_system_create(ctx, gm.grid, 0)
        out["analysis_s"] = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
            part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
            cells = gm.grid.active_cells()
            n = len(cells)
            ps = np.empty(n, np.int32)
            Ms = ms.ms_partition_components(ctx, s, part * 2 + gm.facies[cells].astype(np.int32), ps)
            q = torch.from_numpy(gm.q_active()).to(dev)
            for prec, nm in ((ms.MS_PREC_FP64, "fp64"), (ms.MS_PREC_MIXED, "mixed")):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b1, it1 = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
                b2, it2 = ms.ms_build_basis(ctx, s, ps, Ms, support=ms.MS_SUPPORT_HOP, precision=prec)
                c1, c2 = ms.ms_galerkin(ctx, s, b1, prec), ms.ms_galerkin(ctx, s, b2, prec)
                torch.cuda.synchronize()
                setup = time.perf_counter() - t0
                res = {"setup_s": setup, "basis_iters": [it1, it2], "coarse_blocks": [M, Ms]}
                for outer, key, sched in ((ms.MS_OUTER_GMRES, "gmres", 0), (ms.MS_OUTER_RICHARDSON, "richardson_dp_inf", 2)):
                    p = torch.zeros_like(q)
                    ms.ms_solve(ctx, s, [c1, c2], q, p, tol=1e-6, max_iter=3000, precision=prec, outer=outer,
                                adapt_schedule=sched)   # warm-up (workspaces)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    p.zero_()
                    e0.record(stream)
                    info = ms.ms_solve(ctx, s, [c1, c2], q, p, tol=1e-6, max_iter=3000, precision=prec, outer=outer,
                                       adapt_schedule=sched)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    t = e0.elapsed_time(e1)
                    res[key] = {"iters": info["iters"], "converged": info["converged"], "solve_ms": t,
                                "solve_unknowns_per_s": n / (t * 1e-3), "rel_residual": info["rel_residual"]}
                out[nm] = res
                for h in (c1, c2):
                    ms.ms_coarse_release(h)
                for h in (b1, b2):
                    ms.ms_basis_release(h)
        ms.ms_system_release(s)
    finally:
        ms.ms_destroy(ctx)
    return out


def run_ensemble(args, emit=True):
    """Ensemble step: for every member, basis re-smoothing + Galerkin + solve,
    all members in one ms_solve_batch call (members overlap on worker streams);
    the same work with one worker is timed beside it."""
    rank, world, local = dist_env()
    import torch
    import numpy as np
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import geomodel as G
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(local, stream)
    prec = ms.MS_PREC_MIXED
    mem = []
    for m in R.member_indices(rank, args.members):
        gm = G.ensemble_member(m)
        s = ms.ms_system_create(ctx, gm.grid, 0)
        ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
        part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
        b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec)
        c = ms.ms_galerkin(ctx, s, b, prec)
        q = torch.from_numpy(gm.q_active()).to(dev)
        mem.append(dict(sys=s, stages=[c], q=q, p=torch.zeros_like(q), rebuild=b, n=q.numel(), gm=gm))
    cells = sum(m["n"] for m in mem)
    batch = [dict(sys=m["sys"], stages=m["stages"], q=m["q"], p=m["p"], rebuild=m["rebuild"]) for m in mem]

    def step(workers):
        return ms.ms_solve_batch(ctx, batch, tol=1e-6, max_iter=5000, precision=prec, n_workers=workers,
                                 outer=ms.MS_OUTER_GMRES, restart=30)

    def timed(workers, K):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = [step(workers) for _ in range(K)]
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        if world > 1:
            t = R.max_over_ranks(dist, [t], dev)[0]
        return t, outs[-1]

    # work-item shape of the batched basis smoothing: cached per device, tuned once
    from paper_2001_01624_gb300 import autotune
    tuning = autotune.tuned(ctx, [m["sys"] for m in mem], [m["rebuild"] for m in mem], local, workload="ensemble")
    for _ in range(args.warmup):
        step(args.workers)
    ms.ms_profile_reset()
    sampler = ClockSampler(local)
    sampler.start()
    t_par, out = timed(args.workers, args.steps)
    clocks = sampler.stop()
    launches = ms.ms_profile_read()["_total_launches"]
    t_seq, _ = timed(1, 1)
    # traced step for per-kernel durations, on one worker so that a launch's
    # events time that launch alone (with concurrent members they also time
    # the others): the GPU time of each kernel family over the whole ensemble
    ms.ms_profile_reset()
    ms.ms_profile_enable(True)
    step(1)
    torch.cuda.synchronize()
    ms.ms_profile_enable(False)
    prof = ms.ms_profile_read()
    prof.pop("_total_launches")
    kernels = {k: v for k, v in prof.items() if v["timed_launches"] > 0}
    # the roofline of the batched smoothing (one persistent launch over every
    # member), else of the kernel family with the most GPU time
    dom = ("msrsb_batch32" if "msrsb_batch32" in kernels else
           max(kernels, key=lambda k: kernels[k]["total_ms"]))
    gpu_ms = sum(v["total_ms"] for v in kernels.values())
    top = {k: {"launches": v["timed_launches"], "ms": round(v["total_ms"], 2)}
           for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["total_ms"])[:12]}
    dk = kernels[dom]
    peak, peak_src = measured_peak()
    avg_ms = dk["total_ms"] / dk["timed_launches"]
    bytes_launch = dk["bytes"] / dk["timed_launches"]
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9 if bytes_launch else 0.0
    K = args.steps
    value = cells * K * world / (t_par * 1e-3)
    cyc = [o["iters"] for o in out]
    line = {
        "metric": "fine-cell unknowns/sec to 1e-6 rel residual (ensemble: basis + Galerkin + solve per member)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_par / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 bulk + f64 residual/refinement", "data": "synthetic",
        "config": {"workload": ENSEMBLE.format(m=args.members), "members": args.members, "cells": cells,
                   "workers": args.workers, "parallelism": "replicas (one ensemble slice per GPU)",
                   "batch_tuning": {"tile_cells": tuning["tile_cells"], "ctas_per_sm": tuning["ctas_per_sm"]},
                   "l2": "no flush: the step's working set (all members) exceeds the 129 MB L2"},
        "sequential": {"value": cells * world / (t_seq * 1e-3), "ms_per_step": t_seq, "workers": 1},
        "members": {"converged": sum(o["converged"] for o in out), "cycles_min": min(cyc), "cycles_max": max(cyc),
                    "cycles_mean": sum(cyc) / len(cyc)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs", "traffic": ncu_traffic(dom),
                     "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_ms,
                     "timing": "CUDA events around every launch of one traced step on one worker"},
        "gpu_time": {"kernels_ms": gpu_ms, "top": top,
                     "note": "summed device time of every launch of one step, members one after another"},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_e2e:
        qh = [torch.from_numpy(m["gm"].q_active()).pin_memory().numpy() for m in mem]
        ph = [torch.zeros(m["n"], dtype=torch.float64).pin_memory().numpy() for m in mem]
        hb = [dict(sys=m["sys"], stages=m["stages"], q=q, p=p, rebuild=m["rebuild"]) for m, q, p in zip(mem, qh, ph)]
        ms.ms_solve_batch(ctx, hb, tol=1e-6, max_iter=5000, precision=prec, n_workers=args.workers,
                          outer=ms.MS_OUTER_GMRES, restart=30)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            ms.ms_solve_batch(ctx, hb, tol=1e-6, max_iter=5000, precision=prec, n_workers=args.workers,
                              outer=ms.MS_OUTER_GMRES, restart=30)
        torch.cuda.synchronize()
        e2e = time.perf_counter() - t0
        line["e2e"] = {"value": cells * K * world / e2e, "unit": UNIT,
                       "h2d_bytes_per_step": int(sum(q.nbytes for q in qh)),
                       "d2h_bytes_per_step": int(sum(p.nbytes for p in ph)), "ms_per_step": 1e3 * e2e / K}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = ensemble_oracle_sample(mem, out)
    for m in mem:
        ms.ms_coarse_release(m["stages"][0])
        ms.ms_basis_release(m["rebuild"])
        ms.ms_system_release(m["sys"])
    ms.ms_destroy(ctx)
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


SERVING = ("serving: Poisson arrivals (mean {rate:g} req/s, {req} requests, seed 7) of sequential-implicit two-phase "
           "time steps (Corey n = 2, mu_w = 1, mu_o = 3 cP, porosity 0.2; 0.2 % of the pore volume injected per step) on "
           "{m} resident geomodels of N log-uniform in [50k, 2M] cells (lognormal, sigma 2, correlation 8 cells, "
           "Kz = 0.1 Kx; 10x10x5 coarse blocks); per request: total mobility, TPFA assembly with upstream face "
           "mobility, Galerkin re-formed on the resident basis, dynamic stage from the last pressure change, "
           "mixed-precision GMRES(30) with the multistage cycle as preconditioner from the previous pressure to "
           "1e-6, CFL-limited upstream transport; "
           "{w} worker slots (continuous batching)")


def serving_models(m_count, torch, dev, seed=0):
    from paper_2001_01624_gb300 import geomodel as G, serve
    rng = np.random.default_rng(seed)
    models = []
    for k in range(m_count):
        N = float(np.exp(rng.uniform(np.log(5e4), np.log(2e6))))
        nz = int(rng.integers(20, 61))
        nxy = max(10, int(round(np.sqrt(N / nz))))
        nx = max(10, int(round(nxy * rng.uniform(0.6, 1.4))))
        ny = max(10, int(round(N / nz / nx)))
        gm = G.lognormal_box(nx, ny, nz, seed=2000 + k, sigma=2.0, corr=8.0, block=(10, 10, 5), kz_ratio=0.1)
        gm.q[:] *= 1e-4
        models.append(serve.Model(k, gm, torch, dev))
    return models


def run_serving(args, emit=True):
    rank, world, local = dist_env()
    import torch
    global np
    import numpy as np
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import serve
    models = serving_models(args.models, torch, dev, seed=R.serving_seed(rank))

    def dt_of(mid):
        m = models[mid]
        vol = m.gm.grid.dx * m.gm.grid.dy * m.gm.grid.dz
        return 0.002 * 0.2 * vol * m.n / 1e-4
    srv = serve.Server(torch, dev, models, workers=args.workers)
    srv.warm(0.0)
    ms.ms_profile_reset()
    reqs = serve.poisson_stream(args.requests, args.rate, len(models), dt_of, seed=7 + rank)
    sampler = ClockSampler(local)
    sampler.start()
    srv.run(reqs)
    clocks = sampler.stop()
    launches = ms.ms_profile_read()["_total_launches"]
    st = serve.latency_stats(reqs)
    if world > 1:
        st["p99_ms"], st["p50_ms"] = R.max_over_ranks(dist, [st["p99_ms"], st["p50_ms"]], dev)
    cells = sum(models[r.model].n for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    # the same server under a load it can sustain: Poisson arrivals at 70 % of the
    # throughput just measured, so that the latencies are service, not queueing
    rate2 = 0.7 * st["throughput_req_s"]
    n2 = int(min(args.requests, max(40, 12.0 * rate2)))
    reqs2 = serve.poisson_stream(n2, rate2, len(models), dt_of, seed=11 + rank)
    srv.run(reqs2)
    st2 = serve.latency_stats(reqs2)
    if world > 1:
        st2["p99_ms"], st2["p50_ms"] = R.max_over_ranks(dist, [st2["p99_ms"], st2["p50_ms"]], dev)
    line = {"metric": "p99 request latency (serving: arrival to result on the host)", "value": st["p99_ms"],
            "unit": "ms", "n_gpus": world, "steps": args.requests, "warmup": 1, "ms_per_step": st["mean_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 bulk + f64 residual/refinement", "data": "synthetic",
            "config": {"workload": SERVING.format(rate=args.rate, req=args.requests, m=args.models, w=args.workers),
                       "models": args.models, "cells_resident": sum(m.n for m in models),
                       "parallelism": "replicas (one stream of requests per GPU)"},
            "latency": st,
            "requests": {"cycles_mean": float(np.mean([r.cycles for r in reqs])),
                         "cycles_max": int(max(r.cycles for r in reqs)),
                         "substeps_mean": float(np.mean([r.substeps for r in reqs])),
                         "max_rel_residual": float(max(r.rel_residual for r in reqs)),
                         "unknowns_per_s": cells * world / span},
            "sustained_load": {"rate_req_s": rate2, "requests": n2, "p50_ms": st2["p50_ms"], "p99_ms": st2["p99_ms"],
                               "mean_ms": st2["mean_ms"], "throughput_req_s": st2["throughput_req_s"]},
            "gpu_launches": int(launches), "clocks": clocks}
    srv.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def ensemble_oracle_sample(mem, out):
    """CPU oracle on the two smallest members: setup in full, 10 basis
    iterations and 10 cycles timed and scaled to each member's measured counts;
    the unknowns/s of the sample is reported for the ensemble."""
    import oracle as O
    O.build()
    idx = sorted(range(len(mem)), key=lambda k: mem[k]["n"])[:2]
    secs = cells = 0.0
    for k in idx:
        gm = mem[k]["gm"]
        t0 = time.perf_counter()
        s = O.assemble_tpfa(gm.grid, gm.perm)
        Ap, qp = O.pin(s.A, gm.q_active(), 0)
        part, M = O.partition_cartesian(gm.grid, s.cells, gm.block)
        sp, sc = O.support_box(gm.grid, s.cells, s.A, part, M, gm.block)
        fixed = time.perf_counter() - t0
        t0 = time.perf_counter()
        B = O.msrsb_basis(s.A, part, M, sp, sc, 2.0 / 3.0, 0.0, 10)
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        L = O.cholesky(O.galerkin(Ap, B))
        lu = O.ilu0(Ap)
        fixed += time.perf_counter() - t0
        t0 = time.perf_counter()
        O.ms_gmres(Ap, [(B, L)], qp, tol=0.0, max_iter=10, restart=30, lu=lu)
        ts = time.perf_counter() - t0
        secs += fixed + tb * out[k]["basis_iters"] / 10 + ts * out[k]["iters"] / 10
        cells += mem[k]["n"]
    return {"value": cells / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle (plain C, FP64, 1 thread) on the 2 smallest members ({int(cells)} cells): setup in "
                      f"full, 10 basis iterations and 10 GMRES(30) steps timed, scaled to each member's GPU "
                      f"iteration counts"}


def run_profile_ilu(args):
    """ILU(0) applications alone on the 60x220xNZ geomodel, or the faulted
    200x200x50 one (untimed)."""
    import torch
    import numpy as np
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import geomodel as G
    dev = torch.device("cuda:0")
    if args.faulted:
        gm = G.config3(0)
    else:
        gm = G.config2(0) if args.nz == 85 else G.lognormal_box(60, 220, args.nz, seed=0, block=(10, 20, 5),
                                                                 kz_ratio=0.1)
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(0, stream)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    with torch.cuda.stream(stream):
        ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
        r = torch.from_numpy(gm.q_active()).to(dev)
        z = torch.zeros_like(r)
        for prec in (ms.MS_PREC_FP64, ms.MS_PREC_MIXED):
            for _ in range(args.profile_ilu):
                ms.ms_ilu_apply(ctx, s, r, z, prec)
    torch.cuda.synchronize()
    ms.ms_system_release(s)
    ms.ms_destroy(ctx)
    return 0


def run_profile_coarse_sweep(args):
    """Galerkin coarse operators of the 60x220x85 geomodel in FP64 and mixed
    precision: the coarse inverse by the FP64 sweep and by the tensor-core
    sweep (untimed; for ncu captures)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import geomodel as G
    dev = torch.device("cuda:0")
    gm = G.config2(0)
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(0, stream)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    with torch.cuda.stream(stream):
        ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
        part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
        for prec in (ms.MS_PREC_FP64, ms.MS_PREC_MIXED):
            b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block, precision=prec, max_iter=20)
            c = ms.ms_galerkin(ctx, s, b, prec)
            ms.ms_coarse_release(c)
            ms.ms_basis_release(b)
    torch.cuda.synchronize()
    ms.ms_system_release(s)
    ms.ms_destroy(ctx)
    return 0


def run_profile_coarse(args):
    """The finite-volume coarse stage of the 60x220x85 geomodel alone (untimed)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import geomodel as G
    dev = torch.device("cuda:0")
    gm = G.config2(0)
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(0, stream)
    s = ms.ms_system_create(ctx, gm.grid, 0)
    with torch.cuda.stream(stream):
        ms.ms_assemble_tpfa(ctx, s, torch.from_numpy(gm.perm.ravel().copy()).to(dev))
        part, M = ms.ms_partition_cartesian(ctx, s, gm.block)
        b, _ = ms.ms_build_basis(ctx, s, part, M, block=gm.block)
        c = ms.ms_coarse_create(ctx, s, b, ms.MS_PREC_FP64, ms.MS_RESTRICT_FV)
    torch.cuda.synchronize()
    ms.ms_coarse_release(c)
    ms.ms_basis_release(b)
    ms.ms_system_release(s)
    ms.ms_destroy(ctx)
    return 0


def run_coupling(args):
    """Coupling-strength study (dynamic bases against the viscosity ratio):
    average Richardson cycles per pressure solve for the general stage alone,
    Dp(1) and Dp(Inf), 40 sequential two-phase steps per run."""
    import torch
    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return 0
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import coupling as CP
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = ms.ms_create(local, stream)
    steps = 40
    CP.study(ctx, ratios=(2.0,), steps=3)                      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows = CP.study(ctx, steps=steps)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    ms.ms_destroy(ctx)
    solves = len(rows) * len(CP.SCHEDULES) * steps
    line = {"metric": "pressure solves per second (coupling study, 42x22, Richardson to 1e-6)",
            "value": solves / secs, "unit": "solves/s", "n_gpus": 1, "steps": steps, "warmup": 1,
            "higher_is_better": True, "scaling": "replicas", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "coupling study: 42x22 lognormal (sigma 2, correlation 8 cells), 6x2 general "
                                   "blocks, injector / producer columns, linear relative permeabilities, "
                                   "1 PV in 40 steps; mu_w/mu_o in 1/50..50"},
            "avg_cycles_per_solve": rows, "seconds": secs}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_ilu:
        return run_profile_ilu(args)
    if args.profile_coarse:
        return run_profile_coarse(args)
    if args.profile_coarse_sweep:
        return run_profile_coarse_sweep(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "coupling":
        return run_coupling(args)
    import torch
    import numpy as np
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2001_01624_gb300 as ms
    from paper_2001_01624_gb300 import geomodel as G

    gm = G.config2(R.geomodel_seed(rank))
    stream = torch.cuda.Stream(dev)
    ctx = ms.ms_create(local, stream)
    if args.profile_steps and args.profile_mixed:
        plan = Plan(ms, ctx, gm, ms.MS_PREC_MIXED, dev, torch)
        for _ in range(args.profile_steps):
            plan.step()
        torch.cuda.synchronize()
        return 0
    precs = [ms.MS_PREC_FP64] + ([] if args.no_mixed else [ms.MS_PREC_MIXED])
    plans = {p: Plan(ms, ctx, gm, p, dev, torch) for p in precs}
    n = plans[ms.MS_PREC_FP64].n

    if args.profile_steps:
        for _ in range(args.profile_steps):
            plans[ms.MS_PREC_FP64].step()
        torch.cuda.synchronize()
        return 0

    results = {}
    rich = {}
    clocks = None
    for prec, plan in plans.items():
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                plan.step()
        # timed region (tracing off; launch counts are still kept)
        ms.ms_profile_reset()
        sampler = ClockSampler(local) if prec == ms.MS_PREC_FP64 else None
        if sampler:
            sampler.start()
        ms_tot, infos = timed_steps(torch, plan, stream, args.steps, dist, world)
        if sampler:
            clocks = sampler.stop()
        counts = ms.ms_profile_read()
        # traced step: every launch timed with a pair of CUDA events on its stream,
        # for the per-kernel durations
        ms.ms_profile_reset()
        ms.ms_profile_enable(True)
        plan.step()
        torch.cuda.synchronize()
        ms.ms_profile_enable(False)
        prof = ms.ms_profile_read()
        results[prec] = dict(ms=ms_tot, infos=infos, prof=prof, launches=counts["_total_launches"])
        # the same step with Richardson cycles (run as one CUDA graph per solve)
        with torch.cuda.stream(stream):
            plan.step(outer="richardson")
        r_ms, r_infos = timed_steps(torch, plan, stream, max(1, args.steps // 2), dist, world, outer="richardson")
        rich[prec] = dict(ms=r_ms, infos=r_infos, steps=max(1, args.steps // 2))

    r64 = results[ms.MS_PREC_FP64]
    K = args.steps
    value = n * K * world / (r64["ms"] * 1e-3)
    prof = r64["prof"]
    prof.pop("_total_launches")
    launches = r64["launches"]
    # dominant kernel (by device time) and its roofline
    kernels = {k: v for k, v in prof.items() if v["timed_launches"] > 0}
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    dk = kernels[dom]
    peak, peak_src = measured_peak()
    units = dk["timed_launches"]
    if dom == "msrsb":
        # smoothing iterations are enqueued in batches: the launches after convergence
        # do nothing, so per-launch figures divide the whole time by the iterations done
        units = r64["infos"][-1]["basis_iters"]
    avg_ms = dk["total_ms"] / units
    bytes_launch = dk["bytes"] / dk["timed_launches"]
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom)
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs", "traffic": traffic,
            "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_ms, "launches": dk["timed_launches"],
            "iterations": units,
            "timing": "CUDA events around every launch of one traced step of the same workload"}
    if dom == "msrsb":
        # FP64 basis smoothing is bound by the FP64 pipe (ncu: 88 % busy, DRAM 16 %).  Per basis entry,
        # with the rows prescaled by omega / A_ii once per smoothing run: one multiply for the diagonal,
        # W multiply-adds for the neighbours, the renormalisation's sum and scale = 2 W + 3 flops
        plan = plans[ms.MS_PREC_FP64]
        W = ms.ms_system_get_info(plan.sys)["ell_width"]
        nnz = ms.ms_basis_get_info(plan.basis)["nnz"]
        flops = nnz * (2 * W + 3)
        tf = flops / (avg_ms * 1e-3) / 1e12
        roof.update({"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": tf / FP64_PEAK_TFLOPS, "peak_source": "nominal FP64 of the GB300 (1.25 TFLOP/s)",
                     "algorithmic_flops_per_launch": flops,
                     "hbm": {"achieved_gbs": achieved, "frac_of_measured": achieved / peak}})
    info0 = r64["infos"][-1]
    solve_ms = info0["seconds"] * 1e3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": r64["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": n, "coarse_blocks": plans[ms.MS_PREC_FP64].M,
                   "precision": "fp64", "parallelism": "replicas (one independent seeded geomodel per GPU)",
                   "l2": "no flush: working set of each step (A, ILU factors, 8-slot basis, vectors) exceeds the "
                         "129 MB L2"},
        "solve": {"outer": "GMRES(30), multistage cycle as right preconditioner", "steps": info0["iters"],
                  "basis_iters": info0["basis_iters"], "rel_residual": info0["rel_residual"], "solve_ms": solve_ms,
                  "solve_unknowns_per_s": n / (solve_ms * 1e-3)},
        "roofline": roof,
        "kernels": {k: {"launches": v["timed_launches"], "ms": round(v["total_ms"], 3),
                        "share": round(v["total_ms"] / sum(x["total_ms"] for x in kernels.values()), 4),
                        "GBps": (round(v["bytes"] / (v["total_ms"] * 1e-3) / 1e9, 1) if v["bytes"] else None)}
                    for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["total_ms"])},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    line["richardson"] = {}
    for prec, nm in ((ms.MS_PREC_FP64, "fp64"), (ms.MS_PREC_MIXED, "mixed")):
        if prec in rich:
            rr = rich[prec]
            ir = rr["infos"][-1]
            line["richardson"][nm] = {"value": n * rr["steps"] * world / (rr["ms"] * 1e-3), "unit": UNIT,
                                      "ms_per_step": rr["ms"] / rr["steps"], "cycles": ir["iters"],
                                      "solve_ms": ir["seconds"] * 1e3, "rel_residual": ir["rel_residual"]}
    if ms.MS_PREC_MIXED in results:
        rm = results[ms.MS_PREC_MIXED]
        im = rm["infos"][-1]
        pk = {k: v for k, v in rm["prof"].items() if k != "_total_launches" and v["timed_launches"] > 0}
        tot = sum(v["total_ms"] for v in pk.values())
        line["mixed"] = {"value": n * K * world / (rm["ms"] * 1e-3), "unit": UNIT, "ms_per_step": rm["ms"] / K,
                         "dtype": "f32 bulk + f64 residual/refinement", "steps": im["iters"],
                         "basis_iters": im["basis_iters"], "solve_ms": im["seconds"] * 1e3,
                         "rel_residual": im["rel_residual"],
                         "kernels": {k: {"launches": v["timed_launches"], "ms": round(v["total_ms"], 3),
                                         "share": round(v["total_ms"] / tot, 4)}
                                     for k, v in sorted(pk.items(), key=lambda kv: -kv[1]["total_ms"])[:10]}}
        cinv = ms.ms_coarse_get_inverse(ctx, plans[ms.MS_PREC_MIXED].coarse)
        ck = rm["prof"].get("coarse_sweep_tc") or {}
        line["mixed"]["coarse"] = {"inverse": "fp64" if cinv["fp64"] else "fp32 (tensor cores)",
                                   "fp32_check": cinv["inv_error"], "refine_steps": cinv["refine_steps"],
                                   "sweep_tc_ms": (ck["total_ms"] / ck["timed_launches"]) if ck.get("timed_launches")
                                   else None}
        pm = plans[ms.MS_PREC_MIXED].p.cpu().numpy()
        p64 = plans[ms.MS_PREC_FP64].p.cpu().numpy()
        line["mixed"]["rel_err_vs_fp64"] = float(np.linalg.norm(pm - p64) / np.linalg.norm(p64))

    # finite-volume restriction (R sums each block's cells, Sec. 5) on the same
    # basis: A_c = R A P inverted by Gauss-Jordan, GMRES(30), FP64
    if not args.no_fv:
        plan = plans[ms.MS_PREC_FP64]
        cfv = ms.ms_coarse_create(ctx, plan.sys, plan.basis, ms.MS_PREC_FP64, ms.MS_RESTRICT_FV)
        with torch.cuda.stream(stream):
            plan.step(coarse=cfv)
        kf = max(1, args.steps // 2)
        f_ms, f_infos = timed_steps(torch, plan, stream, kf, dist, world, coarse=cfv)
        ms.ms_profile_reset()
        ms.ms_profile_enable(True)
        plan.step(coarse=cfv)
        torch.cuda.synchronize()
        ms.ms_profile_enable(False)
        pf = ms.ms_profile_read()
        fi = f_infos[-1]

        def per_launch(d, k):
            v = d.get(k)
            return None if not v or not v["timed_launches"] else v["total_ms"] / v["timed_launches"]
        line["fv"] = {"value": n * kf * world / (f_ms * 1e-3), "unit": UNIT, "ms_per_step": f_ms / kf,
                      "restriction": "finite volume (block sums)", "steps": fi["iters"],
                      "solve_ms": fi["seconds"] * 1e3, "rel_residual": fi["rel_residual"],
                      "gauss_jordan_ms": per_launch(pf, "coarse_gauss_jordan"),
                      "cholesky_inverse_ms": per_launch(prof, "coarse_sweep64"),
                      "restrict_ms": per_launch(pf, "restrict"), "restrict_galerkin_ms": per_launch(prof, "restrict")}
        ms.ms_coarse_release(cfv)

    # CPR pressure stage (Sec. 4 quasi-IMPES) of a compressible two-phase step on the same grid and basis:
    # J* and r* from the per-cell state, Galerkin stage of the non-symmetric J* (Gauss-Jordan inverse),
    # GMRES(30) predictor solve to 1e-6
    if not args.no_cpr:
        plan = plans[ms.MS_PREC_FP64]
        pn = plan.p / torch.clamp(plan.p.abs().max(), min=1e-300)
        p_c = 2e7 + 1e6 * pn
        s_c = torch.clamp(0.5 * (1.0 + pn), 0.0, 1.0)
        p0_c = p_c - 1e4
        s0_c = 0.99 * s_c
        qw_c = torch.clamp(plan.q, min=0.0) * 10.0
        qo_c = torch.clamp(plan.q, max=0.0) * 8.0
        rhs_c = torch.empty_like(p_c)
        dp_c = torch.zeros_like(p_c)
        fl = ms.cpr_fluid()
        with torch.cuda.stream(stream):
            ms.ms_cpr_pressure_system(ctx, plan.sys, plan.perm, fl, p_c, s_c, p0_c, s0_c, qw_c, qo_c, 86400.0, rhs_c)
            ccpr = ms.ms_galerkin(ctx, plan.sys, plan.basis, ms.MS_PREC_FP64)

            def cpr_step():
                ms.ms_cpr_pressure_system(ctx, plan.sys, plan.perm, fl, p_c, s_c, p0_c, s0_c, qw_c, qo_c, 86400.0,
                                          rhs_c)
                ms.ms_coarse_refresh(ctx, plan.sys, ccpr)
                dp_c.zero_()
                return ms.ms_solve(ctx, plan.sys, [ccpr], rhs_c, dp_c, tol=1e-6, max_iter=5000,
                                   precision=ms.MS_PREC_FP64, outer=ms.MS_OUTER_GMRES, restart=30)
            cpr_step()
            kc = max(1, args.steps // 2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cinfo = [cpr_step() for _ in range(kc)]
            e1.record(stream)
            torch.cuda.synchronize()
            c_ms = e0.elapsed_time(e1)
            ms.ms_profile_reset()
            ms.ms_profile_enable(True)
            cpr_step()
            torch.cuda.synchronize()
            ms.ms_profile_enable(False)
            pc = ms.ms_profile_read()
        ms.ms_coarse_release(ccpr)

        def stat(k):
            v = pc.get(k)
            if not v or not v["timed_launches"]:
                return None
            t = v["total_ms"] / v["timed_launches"]
            return {"ms": t, "GBps": (v["bytes"] / v["timed_launches"]) / (t * 1e-3) / 1e9 if v["bytes"] else None}
        line["cpr"] = {"value": n * kc * world / (c_ms * 1e-3), "unit": UNIT, "ms_per_step": c_ms / kc,
                       "stage": "CPR pressure system (quasi-IMPES) + Galerkin + GJ inverse + GMRES(30) to 1e-6",
                       "steps": cinfo[-1]["iters"], "rel_residual": cinfo[-1]["rel_residual"],
                       "cpr_cell": stat("cpr_cell"), "cpr_rows": stat("cpr_rows"),
                       "gauss_jordan_ms": (stat("coarse_gauss_jordan") or {}).get("ms")}

    # end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        plan = plans[ms.MS_PREC_FP64]
        perm_h = torch.from_numpy(gm.perm.ravel().copy()).pin_memory().numpy()
        q_h = torch.from_numpy(gm.q_active()).pin_memory().numpy()
        p_h = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
        plan.step(perm_h, q_h, p_h)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            plan.step(perm_h, q_h, p_h)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            e2e_s = R.max_over_ranks(dist, [e2e_s], dev)[0]
        line["e2e"] = {"value": n * K * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(perm_h.nbytes + q_h.nbytes),
                       "d2h_bytes_per_step": int(p_h.nbytes), "ms_per_step": 1e3 * e2e_s / K}

    # CPU oracle baseline (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build(openmp=True)
        line["cpu_baseline"] = cpu_baseline_line(n, oracle_full_step(gm))
        if args.oracle_single:
            line["cpu_baseline"]["single_thread"] = cpu_baseline_line(n, oracle_full_step(gm, openmp=False))

    for p in plans.values():
        p.release()
    ms.ms_destroy(ctx)
    # the other configurations, compactly (N = 1 only): faulted c3 solves,
    # the batched ensemble, the serving stream
    if rank == 0 and world == 1 and not args.no_extras:
        line["c3"] = c3_extra(torch, ms, G, dev, stream)
        ea = argparse.Namespace(**vars(args))
        ea.steps, ea.warmup, ea.no_e2e, ea.no_cpu_baseline = 2, 1, True, True
        el = run_ensemble(ea, emit=False)
        line["ensemble"] = {k: el[k] for k in ("value", "unit", "ms_per_step", "sequential", "members", "roofline",
                                                "gpu_time")}
        line["ensemble"]["config"] = el["config"]
        sa = argparse.Namespace(**vars(args))
        sa.requests = min(args.requests, 200)
        sl = run_serving(sa, emit=False)
        line["serving"] = {k: sl[k] for k in ("latency", "requests", "sustained_load", "config")}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
