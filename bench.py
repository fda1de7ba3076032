#!/usr/bin/env python
"""Benchmark: cut-cell VEM pressure projection on a 128^3 grid.

Workload: two boxes 0.3 x 0.5 x 0.3, each rotated 17 degrees about z, facing
faces 0.3 cells apart; first-order VEM; 5-level diffusion-free Galerkin
hierarchy; seeded 32-mode Fourier velocity; CG to relative residual 1e-6.
One step = one whole projection (RHS, multigrid-preconditioned CG, velocity
correction) with the velocity already resident on the device.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the single-scene solve has no shard with one exchange step, so N
ranks run N independent replicas (no data-path collective); the time is the
max over ranks.  `--impl reference` times the FP64 CPU oracle instead on a
bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "128^3 cut-cell VEM pressure solve ms to 1e-6 rel resid; V-cycle HBM GB/s vs peak"
# Per-launch DRAM traffic of the level-0 FP32 Chebyshev step at 128^3 from ncu
# captures of the current kernel (one entry per captured launch shape): tuned
# launch shape index, stencil use, template variant, bytes.  A run whose tuned
# shape has no capture reports null traffic.
TRAFFIC_128 = [{"cfg": 0, "stencil": 1, "variant": "k_cheb_step<float, 2, 1, 1, 1> (grid 7700)",
                "bytes": 98826752 + 3104512}]

# Iterations of the coarsest-level CG in the timed solver: the fixed-count CG
# is the method's coarsest solve (the library's and the oracle's default is
# 80); 160 is the count that minimises the time to 1e-6 on this workload with
# the persistent coarsest kernel (measured: 80 / 120 / 160 / 200 iterations
# give 9 / 7 / 6 / 6 outer iterations and 13.1 / 11.8 / 11.4 / 12.7 ms).
BENCH_COARSE_ITERS = 160

WORKLOAD = ("two boxes 0.3x0.5x0.3 rotated 17deg about z, 0.3-cell gap, 128^3 background grid, "
            "first-order VEM, 5 levels, 32-mode Fourier velocity, rel_tol 1e-6, "
            f"{BENCH_COARSE_ITERS} coarsest-level CG iterations")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _oracle_worker(threads, steps, warmup, N_sample):
    """Child process of oracle_sample: the FP64 oracle's set-up and projection
    timings on the sample, with the BLAS / OpenMP pools of this process sized
    by the environment its parent set (printed as one JSON line)."""
    import scenes
    from oracle.pipeline import build_system, project
    sc = scenes.config(1, N_sample)
    t0 = time.perf_counter()
    S = build_system(sc)
    setup_s = time.perf_counter() - t0
    u = sc.velocity(S.meshes[0].V)
    for _ in range(warmup):
        project(S, u, tol=1e-6)
    t = []
    its = 0
    for _ in range(max(1, steps)):
        t1 = time.perf_counter()
        _, _, its, _ = project(S, u, tol=1e-6)
        t.append((time.perf_counter() - t1) * 1e3)
    print(json.dumps({"ms": float(np.median(t)), "iters": its, "ndof": len(S.free[0]), "setup_s": setup_s,
                      "threads": threads}), flush=True)


def oracle_sample(steps, warmup, N_sample=16):
    """FP64 CPU oracle on the same scene at a bounded resolution, measured:
    its set-up (cut cells, hierarchy, elements, Galerkin operators), then the
    median ms per projection (RHS + multigrid PCG to 1e-6 + correction) with
    one BLAS thread and with every host core.  Each thread count runs in a
    fresh process whose thread pools are sized through the environment."""
    ncores = os.cpu_count() or 1
    res = {}
    for threads in (1, ncores):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                  "NUMEXPR_NUM_THREADS"):
            env[k] = str(threads)
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", str(threads),
                              str(steps), str(warmup), str(N_sample)], env=env, check=True,
                             stdout=subprocess.PIPE, text=True).stdout
        res[threads] = json.loads([x for x in out.splitlines() if x.startswith("{")][-1])
    one = res[1]
    return {"ms": one["ms"], "ms_all_cores": res[ncores]["ms"], "cores_all": ncores, "ndof": one["ndof"],
            "iters": one["iters"], "setup_s": one["setup_s"], "N": N_sample}


def cpu_baseline_of(o, ndof_full):
    """The oracle's measured numbers on its sample; the DOF-scaled figure for
    the full workload is an extrapolation and is kept in its own field."""
    return {"value": o["ms"], "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"oracle projection of the same two-box scene at {o['N']}^3 ({o['ndof']} DOFs, "
                      f"{o['iters']} CG iterations), median, 1 BLAS thread; set-up {o['setup_s']:.1f} s untimed "
                      f"in value",
            "all_cores": {"value": o["ms_all_cores"], "cores": o["cores_all"]},
            "setup_s": o["setup_s"],
            "extrapolated_full_workload_ms": o["ms"] * ndof_full / o["ndof"]}


def naive_arm(args, fv, torch, scenes, rank, barrier, max_over_ranks):
    """Ablation (Table 4's "Ours^np"): the two-box projection with the naive
    VEM prolongation of Eq. 16 against the diffusion-free one of Eq. 17, same
    solver otherwise (FP32 V-cycle, FP64 CG to 1e-6): coarse nonzeros, CG
    iterations, set-up and projection time of each."""
    k2 = args.order == 2
    sc = scenes.config(4 if k2 else 1, args.N)
    out = {}
    for name, naive in (("diffusion_free", False), ("naive", True)):
        t0 = time.perf_counter()
        S = fv.Solver(order_k=args.order, levels=5, precision="fp32", rel_tol=1e-6, coarse_iters=BENCH_COARSE_ITERS,
                      naive_prolongation=naive)
        S.build(sc.N, sc.tris)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        q = S.query()
        u = torch.tensor(sc.velocity(S.export_level(0)["V"]).T.copy(), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            S.project(u)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            st = S.project(u)[2]
        e1.record()
        barrier()
        out[name] = {"ms": max_over_ranks(e0.elapsed_time(e1) / args.steps), "iters": st["iters"],
                     "rel_res": st["rel_res"], "nnz": q["nnz"], "n_dofs": q["n_dofs"], "setup_s": round(setup, 2),
                     "coarse_mode32": q["coarse_mode32"]}
        S.close()
    scene = (f"holed 1e-5 sheet, k = 2, {args.N}^3" if k2 else WORKLOAD.replace("128^3", f"{args.N}^3"))
    line = {"metric": f"{args.N}^3 {'sheet (k = 2)' if k2 else 'two-box'} projection ms to 1e-6, naive (Eq. 16) "
                      "vs diffusion-free (Eq. 17) prolongation", "value": out["naive"]["ms"], "unit": "ms",
            "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "dtype": "fp32-vcycle/fp64-cg", "config": {"workload": scene},
            "hierarchies": out,
            "coarse_nnz_ratio": [a / b for a, b in zip(out["naive"]["nnz"], out["diffusion_free"]["nnz"])]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def particles_arm(args, fv, torch, scenes, rank, barrier, max_over_ranks):
    """The particle step around the projection (Sec. 3.2-3.3) on the two-box
    scene: 8 stratified particles per background cube, velocities from the
    scene's Fourier field; per step P2G of the velocity to the level-0
    vertices, the projection (FP32 V-cycle, FP64 CG to 1e-6), the FLIP/PIC
    update (alpha 0.95) and one midpoint RK2 step (dt = half a cell at the
    initial largest particle speed).  Every call goes through the C ABI on
    resident device buffers."""
    sc = scenes.config(1, args.N)
    S = fv.Solver(levels=5, precision="fp32", rel_tol=1e-6, coarse_iters=BENCH_COARSE_ITERS)
    S.build(sc.N, sc.tris)
    if args.host_loop:
        S.set_graphs(False)
    Xh = scenes.particles(args.N, per_axis=2, seed=4242)
    X = torch.tensor(Xh, dtype=torch.float64, device="cuda")
    up = torch.tensor(sc.velocity(Xh.T).T.copy(), dtype=torch.float64, device="cuda")
    del Xh
    cell = S.locate(X)
    live = int((cell >= 0).sum())
    dt = 0.5 / (args.N * float(up.abs().max()))
    names = ("p2g", "project", "g2p", "advect")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    iters = []

    def step(e):
        if e:
            e[0].record()
        u = S.p2g(X, up, cell)
        if e:
            e[1].record()
        _, cellpoly, st = S.project(u)
        if e:
            e[2].record()
        S.g2p(X, cell, u, cellpoly, up, 0.95)
        if e:
            e[3].record()
        S.advect(X, cell, cellpoly, dt)
        if e:
            e[4].record()
        return st

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    barrier()
    n0 = S.launch_count()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(args.steps):
            iters.append(step(ev[k])["iters"])
        torch.cuda.synchronize()
    barrier()
    launches = (S.launch_count() - n0) / args.steps
    parts = {nm: sum(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)) / args.steps
             for i, nm in enumerate(names)}
    total = max_over_ranks(sum(ev[k][0].elapsed_time(ev[k][4]) for k in range(args.steps)) / args.steps)
    line = {"metric": f"particle step ms (P2G + projection + G2P + RK2 advection), two boxes {args.N}^3, "
                      "8 particles per cube", "value": total, "unit": "ms", "higher_is_better": False,
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "dtype": "p2g fp32 / projection fp32-vcycle fp64-cg / g2p, advection fp64",
            "config": {"workload": WORKLOAD.replace("128^3", f"{args.N}^3") + "; particles: 8 per cube "
                       "(stratified, seeded), FLIP alpha 0.95, dt half a cell at the initial largest speed",
                       "particles": int(X.shape[1]), "live_particles": live, "dt": dt},
            "parts_ms": parts, "cg_iters": iters, "gpu_launches": launches,
            "particles_per_s": live / (total * 1e-3), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def reference_arm(args, rank):
    if rank != 0:
        return 0
    o = oracle_sample(args.steps, args.warmup)
    cb = cpu_baseline_of(o, args.ndof_full)
    v = o["ms"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def coarse_entry(q, iters=80):
    """The FP32 coarsest-level CG of the V-cycle (the largest share of the
    step): its form, the build-time device time of one solve, and what bounds
    it.  It runs a fixed number of dependent iterations on an operator that
    stays on chip, so it is latency-bound, not HBM-bound."""
    if q["coarse_mode32"] == "persistent":
        ms = q["coarse_ms_persist"][1]
        bound = ("latency: one grid barrier per CG iteration across %d CTAs; the level's FP32 matrix and each "
                 "CTA's halo stay in shared memory, one launch per solve" % q["persist_ctas"])
    else:
        ms = q["coarse_ms32"]
        bound = "latency: two dependent kernel launches per CG iteration (graph replay)"
    return {"form": q["coarse_mode32"], "ms_per_solve": ms, "iterations": iters,
            "us_per_iteration": ms * 1e3 / iters if ms else None, "n_dofs": q["n_dofs"][-1],
            "nnz": q["nnz"][-1], "bound": bound}


def batch_arm(args, fv, torch, scenes, rank, world, barrier, max_over_ranks):
    """Random-scene batch (resolutions 32..96, 1-4 obstacles): every scene on
    its own context and stream, projected in lockstep by one call, against the
    same contexts projected one after the other (FP32 V-cycle, and plain FP64).
    With N ranks the scenes are sharded (balanced by N^3, no collective on the
    data path) and the batch time is the max over ranks.  Host wall clock
    around synchronous calls (several streams are involved), device idle on
    both sides."""
    from paper_2607_17725_b300.batch import shard_scenes
    every = scenes.batch_scenes(args.batch)
    mine = shard_scenes([sc.N for sc in every], world)[rank]
    scs = [every[i] for i in mine]
    t0 = time.perf_counter()
    solvers, us, keep = [], [], []
    for sc in scs:
        st = torch.cuda.Stream()
        keep.append(st)
        S = fv.Solver(levels=5, precision="fp32", rel_tol=1e-6, stream=st.cuda_stream)
        S.build(sc.N, sc.tris)
        V = S.export_level(0)["V"]
        us.append(torch.tensor(sc.velocity(V).T.copy(), dtype=torch.float64, device="cuda"))
        solvers.append(S)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    ps = [torch.empty(S.info["n_vertices"][0], dtype=torch.float64, device="cuda") for S in solvers]
    cps = [torch.empty((S.info["n_cells"][0], 3, 4), dtype=torch.float64, device="cuda") for S in solvers]

    def seq():
        return [S.project(u, p=p, cellpoly=c)[2] for S, u, p, c in zip(solvers, us, ps, cps)]

    def bat():
        return fv.project_batched(solvers, us, ps=ps, cellpolys=cps)[2]

    def run(f):
        for _ in range(args.warmup):
            f()
        barrier()
        n0 = sum(S.launch_count() for S in solvers)
        t = time.perf_counter()
        for _ in range(args.steps):
            stats = f()
        barrier()
        ms = (time.perf_counter() - t) * 1e3 / args.steps
        return max_over_ranks(ms), stats, (sum(S.launch_count() for S in solvers) - n0) // args.steps

    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms_b, st_b, launches = run(bat)
    ms_s, st_s, _ = run(seq)
    for S in solvers:
        S.set_precision("fp64")
    ms_s64, _, _ = run(seq)
    for S in solvers:
        S.set_precision("fp32")
    ndofs = sum(S.info["n_dofs"][0] for S in solvers)
    line = {
        "metric": f"{len(every)} random cut-cell scenes projected to 1e-6 rel resid, ms per batch",
        "value": ms_b, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_b, "higher_is_better": False, "scaling": "strong", "vs_baseline": None,
        "dtype": "fp32-vcycle/fp64-cg", "data": "synthetic",
        "config": {"workload": f"random scene batch x{len(every)} (N 32..96, 1-4 obstacles)",
                   "rank0_scenes": mine, "rank0_dofs": ndofs, "N": [sc.N for sc in scs],
                   "setup_s": round(setup_s, 2),
                   "parallelism": f"scenes sharded over {world} GPU(s), balanced by N^3",
                   "l2": "no flush; the batch's operators exceed L2"},
        "sequential_ms": ms_s, "speedup_vs_sequential": ms_s / ms_b,
        "sequential_fp64_ms": max_over_ranks(ms_s64), "speedup_vs_sequential_fp64": max_over_ranks(ms_s64) / ms_b,
        "iters": [s["iters"] for s in st_b], "max_rel_res": max(s["rel_res"] for s in st_b),
        "same_iters_as_sequential": [a["iters"] for a in st_b] == [b["iters"] for b in st_s],
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def k2_arm(args, fv, torch, scenes, rank, world, barrier, max_over_ranks):
    """Second-order workload: the holed 1e-5 sheet (tilted 30 degrees, 0.2 x
    0.2 hole) at N^3, k = 2 VEM condensed to the vertex, edge and face DOFs,
    5 levels, seeded 32-mode velocity, CG to 1e-6 with the FP32 V-cycle
    (timed), the same in FP64, and a 1e-11 FP64 solve as the reference of
    both."""
    sc = scenes.config(4, args.N)
    t0 = time.perf_counter()
    S = fv.Solver(order_k=2, levels=5, precision="bf16", rel_tol=1e-6)
    S.build(sc.N, sc.tris)
    if args.host_loop:
        S.set_graphs(False)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    q = S.query()
    V = S.export_level(0)["V"]
    nv, nc, nall = q["n_vertices"][0], q["n_cells"][0], q["n_dofs_all"][0]
    u = torch.tensor(sc.velocity(V).T.copy(), dtype=torch.float64, device="cuda")
    p = torch.empty(nall, dtype=torch.float64, device="cuda")
    cp = torch.empty((nc, 3, 4), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(mode, steps, warmup, prof=False):
        S.set_precision(mode)
        for _ in range(warmup):
            S.project(u, p=p, cellpoly=cp)
        barrier()
        if prof:
            S.set_profiling(True)
        n0 = S.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for _ in range(steps):
            stats.append(S.project(u, p=p, cellpoly=cp)[2])
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = (S.launch_count() - n0) // steps
        prof_d = S.get_profile() if prof else None
        if prof:
            S.set_profiling(False)
        return max_over_ranks(ms), stats, launches, prof_d

    # the mixed-precision forms: FP32 level values, and packed BF16 / FP16
    # level values (FP32 vectors and accumulation); a 16-bit form whose solve
    # does not reach the tolerance is recorded with its status
    res = {}
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for m in ("fp32", "bf16", "fp16"):
            try:
                msm, statsm, launchesm, _ = timed(m, args.steps, args.warmup)
                res[m] = {"ms": msm, "stats": statsm, "launches": launchesm, "p": p.clone(), "status": "ok"}
            except fv.FastVEMError as e:
                res[m] = {"ms": float("inf"), "stats": [{"iters": None}], "launches": None, "p": None,
                          "status": str(e)}
    clocks = clk.summary()
    ms32, stats32, p32 = res["fp32"]["ms"], res["fp32"]["stats"], res["fp32"]["p"]
    # the reported value: the fastest mixed-precision form that converged
    mode = min(res, key=lambda m: res[m]["ms"])
    ms, stats, launches = res[mode]["ms"], res[mode]["stats"], res[mode]["launches"]
    _, _, _, prof = timed(mode, max(2, args.steps // 2), 1, prof=True)
    ms64, stats64, _, _ = timed("fp64", args.steps, args.warmup)
    p64 = p.clone()
    S.set_tolerance(1e-11, 2000)
    S.project(u, p=p, cellpoly=cp)
    pt = p.clone()
    S.set_tolerance(1e-6, 500)
    def err(pm):
        return float(torch.linalg.norm(pm - pt) / torch.linalg.norm(pt)) if pm is not None else None

    err64 = err(p64)
    peak, peak_kind = peaks()
    per_launch_ms = prof["total_ms"] / max(1, prof["launches"])
    achieved = prof["bytes_per_launch"] / (per_launch_ms * 1e-3) / 1e9
    line = {
        "metric": f"{args.N}^3 second-order cut-cell VEM pressure solve ms to 1e-6 rel resid (holed 1e-5 sheet)",
        "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": (f"{mode}-level-values/fp32-vcycle/fp64-cg" if mode != "fp32" else "fp32-vcycle/fp64-cg"),
        "data": "synthetic", "mixed_mode": mode,
        "config": {"workload": f"holed sheet 1e-5 thick, 30 deg about x, 0.2x0.2 hole, {args.N}^3, second-order "
                               f"VEM (cell means condensed), 5 levels, 32-mode Fourier velocity, rel_tol 1e-6",
                   "n_dofs_condensed": q["n_dofs"], "n_dofs_all": q["n_dofs_all"], "nnz": q["nnz"],
                   "n_cells": q["n_cells"], "setup_s": round(setup_s, 2),
                   "setup_split_s": {k: round(v, 2) for k, v in q["setup_s"].items()},
                   "coarse_solve": {"fp64_mode": q["coarse_mode"], "fp32_mode": q["coarse_mode32"]},
                   "cg_loop": "host-driven (profiling)" if args.host_loop else "whole-PCG graph, one launch per solve",
                   "l2": "inputs larger than L2, no flush"},
        "iters": stats[-1]["iters"], "rel_res": stats[-1]["rel_res"],
        "modes": {**{("fp32_vcycle" if m == "fp32" else f"{m}_levels"):
                     {"ms": r["ms"] if r["status"] == "ok" else None, "iters": r["stats"][-1]["iters"],
                      "rel_err_vs_fp64_1e-11": err(r["p"]), "status": r["status"]} for m, r in res.items()},
                  "fp64": {"ms": ms64, "iters": stats64[-1]["iters"], "rel_err_vs_fp64_1e-11": err64}},
        "roofline": {"bound": "hbm", "kernel": "k_cheb_step<float> level 0 (fused SELL SpMV + Chebyshev update), "
                               + {"fp32": "FP32", "bf16": "BF16", "fp16": "FP16"}[mode] + " values",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "bytes_per_launch": prof["bytes_per_launch"],
                     "launches": prof["launches"], "avg_launch_us": per_launch_ms * 1e3},
        "coarse_solve_kernel": coarse_entry(q),
        "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ndof-full", type=int, default=1970922,
                    help="level-0 DOFs of the two-box scene at 128^3, to which the oracle sample is scaled")
    ap.add_argument("--workload", default="projection", choices=["projection", "batch", "k2", "naive", "particles"],
                    help="projection: the two-box 128^3 solve (the headline line); batch: the "
                         "random-scene batch projected in lockstep vs one scene at a time; k2: the "
                         "second-order holed sheet; naive: the two-box solve with the naive prolongation "
                         "of Eq. 16 beside the diffusion-free one; particles: the P2G / projection / G2P / "
                         "advection step with 8 particles per cube")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--order", type=int, default=1, choices=[1, 2],
                    help="VEM order of the naive-prolongation ablation (2: the holed sheet)")
    ap.add_argument("--host-loop", action="store_true",
                    help="run the CG loop from the host (every kernel launched on its own) instead of the "
                         "whole-PCG graph; ncu cannot profile kernel nodes of graphs with conditional nodes")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    import scenes
    import paper_2607_17725_b300 as fv
    from paper_2607_17725_b300 import build as fvbuild
    fvbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    if args.workload == "batch":
        return batch_arm(args, fv, torch, scenes, rank, world, barrier, max_over_ranks)
    if args.workload == "k2":
        return k2_arm(args, fv, torch, scenes, rank, world, barrier, max_over_ranks)
    if args.workload == "naive":
        return naive_arm(args, fv, torch, scenes, rank, barrier, max_over_ranks)
    if args.workload == "particles":
        return particles_arm(args, fv, torch, scenes, rank, barrier, max_over_ranks)

    sc = scenes.config(1, args.N)
    t0 = time.perf_counter()
    S = fv.Solver(levels=5, precision="fp32", rel_tol=1e-6, coarse_iters=BENCH_COARSE_ITERS)
    S.build(sc.N, sc.tris)
    if args.host_loop:
        S.set_graphs(False)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    q = S.query()
    try:  # grid quality (Eq. 19), untimed
        _, rho_grid, n_cut = S.quality(0)
        grid_quality = {"rho_P": rho_grid, "cut_cells": n_cut}
    except fv.FastVEMError as e:
        grid_quality = {"error": str(e)}
    V = S.export_level(0)["V"]
    nv, nc = q["n_vertices"][0], q["n_cells"][0]
    u = torch.tensor(sc.velocity(V).T.copy(), dtype=torch.float64, device="cuda")
    p = torch.empty(nv, dtype=torch.float64, device="cuda")
    cp = torch.empty((nc, 3, 4), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(mode, steps, warmup, prof=False):
        S.set_precision(mode)
        for _ in range(warmup):
            S.project(u, p=p, cellpoly=cp)
        barrier()
        if prof:
            S.set_profiling(True)
        n0 = S.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for _ in range(steps):
            stats.append(S.project(u, p=p, cellpoly=cp)[2])
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = (S.launch_count() - n0) // steps
        prof_d = S.get_profile() if prof else None
        if prof:
            S.set_profiling(False)
        return max_over_ranks(ms), stats, launches, prof_d

    with Clocks(local) as clk:
        ms, stats, launches, _ = timed("fp32", args.steps, args.warmup)
    clocks = clk.summary()
    # the level-0 step's launch time, from events around each launch in a
    # separate run (the event pairs force the host-driven CG loop, so this run
    # is not the timed one)
    _, _, _, prof = timed("fp32", max(2, args.steps // 2), 1, prof=True)
    p_mixed = p.clone()
    ms64, stats64, launches64, _ = timed("fp64", args.steps, args.warmup)
    # FP64 reference solution at a tight tolerance for the error of both forms
    S.set_tolerance(1e-11, 1000)
    S.project(u, p=p, cellpoly=cp)
    p_tight = p.clone()
    S.set_tolerance(1e-6, 500)
    S.set_precision("fp64")
    S.project(u, p=p, cellpoly=cp)
    err64 = float(torch.linalg.norm(p - p_tight) / torch.linalg.norm(p_tight))
    err32 = float(torch.linalg.norm(p_mixed - p_tight) / torch.linalg.norm(p_tight))

    # packed BF16 / FP16 level matrices (FP32 vectors and accumulation, FP64
    # outer CG): a second context created in BF16 mode, tuned for its own
    # products, and switched to FP16 (the plane re-packed from the FP32 copy)
    v16 = {"bf16": None, "fp16": None}
    tune_file = os.environ.pop("FVEM_TUNE_FILE", None)  # the pinned decisions are the FP32 context's
    try:
        SB = fv.Solver(levels=5, precision="bf16", rel_tol=1e-6, coarse_iters=BENCH_COARSE_ITERS)
        SB.build(sc.N, sc.tris)
        pb = torch.empty_like(p)
        cpb = torch.empty_like(cp)
        for m in ("bf16", "fp16"):
            try:
                SB.set_precision(m)
                for _ in range(args.warmup):
                    SB.project(u, p=pb, cellpoly=cpb)
                barrier()
                eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                eb0.record(stream)
                for _ in range(args.steps):
                    stb = SB.project(u, p=pb, cellpoly=cpb)[2]
                eb1.record(stream)
                barrier()
                v16[m] = {"ms": max_over_ranks(eb0.elapsed_time(eb1) / args.steps), "iters": stb["iters"],
                          "rel_err": float(torch.linalg.norm(pb - p_tight) / torch.linalg.norm(p_tight))}
            except fv.FastVEMError as e:
                v16[m] = {"error": str(e)}
        SB.close()
    except fv.FastVEMError as e:
        v16 = {"bf16": {"error": str(e)}, "fp16": {"error": str(e)}}
    finally:
        if tune_file is not None:
            os.environ["FVEM_TUNE_FILE"] = tune_file

    # e2e: host buffers through the C ABI (H2D of u', D2H of p and cellpoly inside)
    S.set_precision("fp32")
    uh = torch.empty((3, nv), dtype=torch.float64, pin_memory=True)
    uh.copy_(u.cpu())
    ph = torch.empty(nv, dtype=torch.float64, pin_memory=True)
    cph = torch.empty((nc, 3, 4), dtype=torch.float64, pin_memory=True)
    for _ in range(args.warmup):
        S.project_host_pinned(uh, ph, cph)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.project_host_pinned(uh, ph, cph)
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps)

    peak, peak_kind = peaks()
    per_launch_ms = prof["total_ms"] / max(1, prof["launches"])
    achieved = prof["bytes_per_launch"] / (per_launch_ms * 1e-3) / 1e9
    # DRAM traffic of one level-0 FP32 step, from an ncu capture (dram__bytes
    # read + write) of the first level-0 k_cheb_step launch of this benchmark
    # at 128^3, with the tuning decisions of a plain run.  Valid only for the
    # kernel variant that was captured; otherwise reported as null.
    traffic = None
    for cap in TRAFFIC_128:
        if (args.N == 128 and q["sell_cfg32"] and q["sell_cfg32"][0] == cap["cfg"]
                and q["stencil_used32"][0] == cap["stencil"]):
            traffic = cap["bytes"]
            break
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32-vcycle/fp64-cg", "data": "synthetic",
        "config": {"workload": WORKLOAD, "coarse_iters": BENCH_COARSE_ITERS, "n_dofs": q["n_dofs"], "nnz": q["nnz"],
                   "n_cells": q["n_cells"],
                   "l2": "inputs larger than L2, no flush: every CG iteration reads the FP64 level-0 "
                         "operator (%.2f GB of values+indices)" % (q["nnz"][0] * 12 / 1e9),
                   "parallelism": f"replicas x{world}", "setup_s": round(setup_s, 2),
                   "cg_loop": "host-driven (profiling)" if args.host_loop else "whole-PCG graph, one launch per solve",
                   "setup_split_s": {k: round(v, 2) for k, v in q["setup_s"].items()},
                   "coarse_solve": {"fp64_mode": q["coarse_mode"], "fp64_build_ms": q["coarse_ms"],
                                    "product_shape": q["coarse_cfg"], "fp32_mode": q["coarse_mode32"],
                                    "fp32_build_ms": [q["coarse_ms32_coop"], q["coarse_ms32"]]},
                   "sell_shapes": {"fp64": q["sell_cfg64"], "fp32": q["sell_cfg32"]},
                   "stencil_slices": {"fp32": q["stencil_slices32"], "used": q["stencil_used32"]},
                   "grid_quality": grid_quality},
        "iters": stats[-1]["iters"], "rel_res": stats[-1]["rel_res"],
        "pressure_rel_err_vs_fp64_tight": err32,
        "modes": {"fp32_vcycle": {"ms": ms, "iters": stats[-1]["iters"], "rel_err": err32},
                  "fp64": {"ms": ms64, "iters": stats64[-1]["iters"], "rel_err": err64,
                           "gpu_launches": launches64},
                  "bf16_levels": v16["bf16"], "fp16_levels": v16["fp16"]},
        "roofline": {"bound": "hbm", "kernel": "k_cheb_step<float> level 0 (fused SELL SpMV + Chebyshev update)",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one level-0 launch "
                                        "at 128^3, variant " + str(cap["variant"])) if traffic else None,
                     "bytes_per_launch": prof["bytes_per_launch"], "launches": prof["launches"],
                     "avg_launch_us": per_launch_ms * 1e3},
        "coarse_solve_kernel": coarse_entry(q, BENCH_COARSE_ITERS),
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 3 * nv * 8,
                "d2h_bytes_per_step": (nv + 12 * nc) * 8},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_of(oracle_sample(3, 1), q["n_dofs"][0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    if len(sys.argv) == 6 and sys.argv[1] == "--oracle-worker":
        _oracle_worker(*(int(a) for a in sys.argv[2:]))
        sys.exit(0)
    sys.exit(main())
