"""Benchmark of the FE solve inside one SIMP/OC optimisation iteration on a 2:1-balanced octree
cantilever mesh (base 48x24x24, three refinement levels along a seeded truss, ~2M elements,
~5.4M unknowns), through the C ABI of libtm.

One step = one optimisation iteration on the fixed mesh: PCG solve of C^T K(rho) C u = f to a
relative residual of 1e-8 (FP32 CG with reliable updates: FP64 true-residual replacement after every
10x reduction, warm-started from the previous u; preconditioner: Jacobi plus a Galerkin coarse
correction on the base-grid lattice applied by a V-cycle), expansion u_full = C u, compliance
sensitivities, the volume-weighted filter of Eq. 5 and the OC update.  Metric: GDOF*iter/s =
unknowns * CG iterations / step seconds; time to tolerance is reported beside it for the chosen
solver, the Jacobi mixed solver and FP64 Jacobi-PCG on the same system from the same warm start.

Arms:
  (default)            the GPU library; prints one JSON line (rank 0).
  --impl reference     the oracle (FP64 CPU Jacobi-PCG on its assembled sparse matrix) timed on
                       the host cores on a bounded sample of the same mesh.
Launch with torchrun for N > 1: every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FE solve time to 1e-8 rel residual, GDOF·iter/s: chosen vs FP64 PCG, 1 GB300"
UNIT = "GDOF*iter/s"
ALGO_BYTES_PER_ELEM_F32 = 60.0     # conn 32 + c_e 4 + x 12 + y 12 (FP32 operator)
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels_apply.cu", "element.cuh", "brick.cuh"):
        with open(os.path.join(ROOT, "paper_1009_4975_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_per_launch():
    """DRAM bytes of one operator application from the committed ncu summary, if it was taken
    on the current kernel source (matching hash); else None."""
    path = os.path.join(ROOT, "profiles", "apply_f32_cantilever_48x24x24_L3.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    kv = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    try:
        return float(kv["dram_bytes_per_application"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            os.unlink(self.path)

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
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(total_ms: float, iters: float, device):
    """Max of the timed milliseconds and sum of the CG iterations over all ranks (identity for one
    process).  Replicas exchange nothing else."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, iters
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    n = torch.tensor([iters], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1009_4975_gb300 as P
    from paper_1009_4975_gb300 import build
    import workloads as W

    build.build()
    w = W.config2()
    d = w.dom
    stream = torch.cuda.current_stream()
    ctx = P.tm_create(local, stream=stream)
    t0 = time.perf_counter()
    info = P.tm_mesh_upload(ctx, d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu,
                            w.penal)
    mesh_s = time.perf_counter() - t0
    perm = P.tm_mesh_tables(ctx)["perm"]
    dev = torch.device("cuda", local)
    Ne, Nn, nfree = info["Ne"], info["Nn"], info["n_free"]
    rho = torch.as_tensor(w.rho[perm], device=dev)
    rho_new = torch.empty_like(rho)
    f = torch.zeros(3 * Nn, dtype=torch.float64, device=dev)
    P.tm_build_rhs(ctx, w.load_nodes, w.load_comp, w.load_val, f)
    u = torch.zeros_like(f)
    uf = torch.zeros_like(f)
    dc = torch.zeros_like(rho)
    dch = torch.zeros_like(rho)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rmin = w.r_min

    precond = P.TM_PRECOND_TWOLEVEL if args.precond == "twolevel" else P.TM_PRECOND_JACOBI

    def step(rho_in, rho_out, prec=P.TM_PREC_MIXED):
        st = P.tm_pcg_solve(ctx, rho_in, f, u, rtol=1e-8, max_iter=200000, precision=prec, check_every=args.check_every,
                            graphs=not args.no_graphs, precond=precond, smooth_sweeps=args.nu)
        P.tm_expand(ctx, u, uf)
        comp = P.tm_sensitivity(ctx, rho_in, uf, dc)
        P.tm_filter(ctx, rho_in, dc, rmin, 0, dch)
        chg = P.tm_oc_update(ctx, rho_in, dch, 0.2, 0.2, 0.5, w.rho_min, rho_out)
        return st, comp, chg

    cur, nxt = rho, rho_new
    for _ in range(args.warmup):
        step(cur, nxt)
        cur, nxt = nxt, cur
    torch.cuda.synchronize()

    # ---- timed region: K steps, device-resident inputs
    clocks = Clocks(local)
    P.tm_profile(ctx, True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    step_ms, iters, comps, solve_ms = [], 0, [], 0.0
    step_iters, step_solve_ms = [], []
    u_first = u.clone()            # warm start of the first timed solve
    rho_first = cur.clone()        # and its design: the FP64 comparison re-solves this system
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, comp, chg = step(cur, nxt)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters += st["iterations"]
        solve_ms += 1e3 * st["seconds"]
        step_iters.append(st["iterations"])
        step_solve_ms.append(1e3 * st["seconds"])
        comps.append(comp)
        cur, nxt = nxt, cur
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    prof = P.tm_profile_read(ctx)
    P.tm_profile(ctx, False)
    total_ms = float(sum(step_ms))
    total_ms_job, iters_job = aggregate(total_ms, float(iters), dev)
    value = nfree * iters_job / (total_ms_job * 1e-3) / 1e9

    # ---- end to end: host (pinned) inputs copied in and results copied out each step
    rho_h = torch.empty(Ne, dtype=torch.float64, pin_memory=True)
    rho_h.copy_(cur.cpu())
    f_h = f.cpu().pin_memory()
    u_h = u.cpu().pin_memory()
    out_rho_h = torch.empty_like(rho_h).pin_memory()
    out_u_h = torch.empty_like(u_h).pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    h2d = rho_h.numel() * 8 + f_h.numel() * 8 + u_h.numel() * 8
    d2h = out_rho_h.numel() * 8 + out_u_h.numel() * 8 + 8
    torch.cuda.synchronize()
    te = time.perf_counter()
    e2e_iters = 0
    for _ in range(e2e_steps):
        cur.copy_(rho_h, non_blocking=True)
        f.copy_(f_h, non_blocking=True)
        u.copy_(u_h, non_blocking=True)
        st, comp, chg = step(cur, nxt)
        out_rho_h.copy_(nxt, non_blocking=True)
        out_u_h.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        e2e_iters += st["iterations"]
        rho_h.copy_(out_rho_h)
        u_h.copy_(out_u_h)
    e2e_s = time.perf_counter() - te
    e2e_value = nfree * e2e_iters / e2e_s / 1e9

    # ---- FP64 Jacobi-PCG on the first timed step's system, same warm start, same tolerance
    u64 = u_first.clone()
    st64 = P.tm_pcg_solve(ctx, rho_first, f, u64, rtol=1e-8, max_iter=args.fp64_iters, precision=P.TM_PREC_FP64,
                          check_every=64, raise_on_error=False)
    uj = u_first.clone()
    stj = P.tm_pcg_solve(ctx, rho_first, f, uj, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                         check_every=64, raise_on_error=False)
    jacobi_mixed = {"iterations": stj["iterations"], "time_to_tolerance_ms": 1e3 * stj["seconds"],
                    "gdof_iter_per_s": nfree * stj["iterations"] / stj["seconds"] / 1e9,
                    "rel_residual": stj["rel_residual"], "converged": stj["status"] == 0}
    fp64 = {"gdof_iter_per_s": nfree * st64["iterations"] / st64["seconds"] / 1e9,
            "ms_per_iter": 1e3 * st64["seconds"] / max(st64["iterations"], 1),
            "iterations": st64["iterations"], "rel_residual": st64["rel_residual"],
            "converged": st64["status"] == 0, "time_to_tolerance_ms": 1e3 * st64["seconds"],
            "chosen_same_system": {"iterations": step_iters[0], "time_to_tolerance_ms": step_solve_ms[0]},
            "jacobi_mixed_same_system": jacobi_mixed,
            "speedup_to_tolerance_chosen_vs_fp64": 1e3 * st64["seconds"] / step_solve_ms[0]}

    if rank != 0:
        return
    solver = dict(precond=precond, smooth_sweeps=args.nu, check_every=args.check_every)
    precision = precision_report(P, ctx, rho_first, f, u_first, u64, solver) if args.reports else None
    batch = batch_report(P, W, solver) if (args.batch and args.reports) else None
    multi = multi_load_report(P, W, ctx, w, rho_first, Nn, solver) if (args.batch and args.reports) else None
    tuned = autotune_report(P, W, ctx, w, rho_first, f, u_first, Nn) if (args.batch and args.reports) else None
    adapt = adaptation_timing(P, ctx, cur, d, Ne, dev) if args.reports else None
    adaptive = (adaptive_report(P, W, w, solver, args.adaptive_iters, args.remesh_every)
                if (args.reports and args.adaptive_iters > 0) else None)
    peak, peak_kind = _peaks()
    a_ms = prof["apply32_ms"] / max(prof["apply32_count"], 1)
    algo = ALGO_BYTES_PER_ELEM_F32 * Ne
    achieved = algo / (a_ms * 1e-3) / 1e9
    traffic = _traffic_per_launch()
    cpu = cpu_baseline(args, w) if (args.cpu_baseline and ws == 1) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (operator and CG vectors; f64 true residuals, solution and reductions)",
        "data": "synthetic (seeded octree truss cantilever)",
        "config": {"workload": w.name, "elements": Ne, "nodes": Nn, "unknowns": nfree,
                   "hanging_nodes": info["n_hanging"], "solver": ("mixed: FP32-operator PCG with reliable updates (FP64 true-residual replacement every 10x "
                   "reduction), rtol 1e-8, warm start; preconditioner " +
                   (f"Jacobi + Galerkin coarse correction on the base-grid lattice (V-cycle, {args.nu} l1-Jacobi sweeps)"
                    if precond == P.TM_PRECOND_TWOLEVEL else "Jacobi")), "step": "solve+expand+sensitivity+filter+OC",
                   "l2": "flushed (512 MB write) before every step", "parallelism": f"replicas x{ws}"},
        "time_to_tolerance_ms": solve_ms / args.steps,
        "cg_iterations_per_step": iters / args.steps,
        "compliance": comps,
        "mesh_upload_s": mesh_s,
        "fp64_pcg": fp64,
        "precision": precision,
        "batch": batch,
        "multi_load": multi,
        "autotune": tuned,
        "adaptation": adapt,
        "adaptive_loop": adaptive,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "roofline": {"bound": "hbm", "kernel": "apply_blocks_kernel<float> (the operator: record-driven blocks "
                     "and 4x4x4 equal-level bricks; the partial sums of shared nodes are read by the CG update)", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes": algo, "avg_ms": a_ms,
                     "launches_timed": prof["apply32_count"]},
        "gpu_launches": prof["launches"],
        "clocks": clk,
        "wall_s": wall,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def precision_report(P, ctx, rho, f, u0, u64, solver):
    """Errors of the chosen and FP64 solvers at the bench tolerance (1e-8) on the first timed
    system, against a solve of the same system to 1e-12 (FP64 residual): energy-norm error of u
    (FP64 operator), relative compliance error, sensitivity error relative to max |dc|.  The
    errors against the oracle's direct solution are measured by the GPU precision tests on
    meshes the oracle factors."""
    import torch
    ref = u0.clone()
    st_ref = P.tm_pcg_solve(ctx, rho, f, ref, rtol=1e-12, max_iter=400000, precision=P.TM_PREC_MIXED,
                            raise_on_error=False, **solver)
    um = u0.clone()
    P.tm_pcg_solve(ctx, rho, f, um, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED, **solver)
    uf = torch.zeros_like(f)
    dc = torch.zeros_like(rho)

    def fields(u):
        P.tm_expand(ctx, u, uf)
        c = P.tm_sensitivity(ctx, rho, uf, dc)
        return c, dc.clone()

    c_ref, dc_ref = fields(ref)
    au = torch.zeros_like(f)
    P.tm_apply_K(ctx, rho, ref, au)
    e_ref = float(torch.dot(ref, au))
    out = {"reference": "mixed solve of the same system to rel. residual 1e-12",
           "reference_rel_residual": st_ref["rel_residual"]}
    for name, u in (("chosen_1e-8", um), ("fp64_1e-8", u64)):
        c, dcu = fields(u)
        e = u - ref
        P.tm_apply_K(ctx, rho, e, au)
        out[name] = {"u_energy_rel_err": abs(float(torch.dot(e, au))) ** 0.5 / e_ref ** 0.5 if e_ref > 0 else None,
                     "compliance_rel_err": abs(c - c_ref) / abs(c_ref),
                     "dc_err_rel_max": float((dcu - dc_ref).abs().max() / dc_ref.abs().max())}
    return out


def batch_report(P, W, solver):
    """Sixteen independent designs of 50k-500k leaves (two-level truss cantilevers, seeds
    100-115), solves with the chosen solver from zero to 1e-8: one after another on one stream
    each, then all at once through tm_pcg_solve_batch.  Throughput = sum of unknowns x iterations
    / wall time."""
    import torch
    works = W.batch_designs()
    items = []
    for w in works:
        d = w.dom
        s = torch.cuda.Stream()
        c = P.tm_create(torch.cuda.current_device(), stream=s)
        info = P.tm_mesh_upload(c, d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu,
                                w.penal)
        perm = P.tm_mesh_tables(c)["perm"]
        rho = torch.as_tensor(w.rho[perm], device="cuda")
        f = torch.zeros(3 * info["Nn"], dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s):
            P.tm_build_rhs(c, w.load_nodes, w.load_comp, w.load_val, f)
        items.append((c, rho, f, info["n_free"]))
    torch.cuda.synchronize()

    def run(batched):
        us = [torch.zeros_like(f) for _, _, f, _ in items]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if batched:
            sts = P.tm_pcg_solve_batch([it[0] for it in items], [it[1] for it in items], [it[2] for it in items], us,
                                       rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED, **solver)
        else:
            sts = [P.tm_pcg_solve(c, rho, f, u, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED, **solver)
                   for (c, rho, f, _), u in zip(items, us)]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        work = sum(n * st["iterations"] for (_, _, _, n), st in zip(items, sts))
        return wall, work, [st["iterations"] for st in sts]

    run(True)   # warm-up: graphs captured, kernels loaded
    seq_s, seq_work, seq_it = run(False)
    bat_s, bat_work, bat_it = run(True)
    for c, _, _, _ in items:
        P.tm_destroy(c)
    return {"designs": len(works), "elements": [int(len(w.leaves)) for w in works],
            "unknowns_total": int(sum(it[3] for it in items)), "iterations": bat_it,
            "same_iterations_as_sequential": bat_it == seq_it,
            "sequential_s": seq_s, "batched_s": bat_s,
            "sequential_gdof_iter_per_s": seq_work / seq_s / 1e9, "batched_gdof_iter_per_s": bat_work / bat_s / 1e9,
            "speedup": seq_s / bat_s}


def multi_load_report(P, W, ctx, w, rho, Nn, solver):
    """Config-4 load cases on the benchmark design: 8 seeded load cases (point loads and face
    tractions on the face x = 2, seeds 10-17) solved from zero to 1e-8 with the chosen solver one
    after another, then in lockstep through tm_pcg_solve_multi (one operator pass, update and
    coarse step for all cases per iteration, CUDA-graph batches)."""
    import torch
    cases = W.load_cases(w.dom, 8, 10)
    dev = rho.device
    F = torch.zeros((len(cases), 3 * Nn), dtype=torch.float64, device=dev)
    for r, (nd, comp, val) in enumerate(cases):
        f = torch.zeros(3 * Nn, dtype=torch.float64, device=dev)
        P.tm_build_rhs(ctx, nd, comp, val, f)
        F[r] = f
    kw = dict(rtol=1e-8, max_iter=200000, precond=solver["precond"], smooth_sweeps=solver["smooth_sweeps"],
              check_every=solver["check_every"])

    def seq():
        its = []
        for r in range(len(cases)):
            u = torch.zeros(3 * Nn, dtype=torch.float64, device=dev)
            its.append(P.tm_pcg_solve(ctx, rho, F[r].contiguous(), u, precision=P.TM_PREC_MIXED, **kw)["iterations"])
        return its

    def lock():
        U = torch.zeros_like(F)
        return [st["iterations"] for st in P.tm_pcg_solve_multi(ctx, rho, F, U, **kw)]

    seq(); lock()                          # warm-up: set-up paths and graphs built once
    torch.cuda.synchronize()
    t0 = time.perf_counter(); it_s = seq(); torch.cuda.synchronize(); seq_s = time.perf_counter() - t0
    t0 = time.perf_counter(); it_l = lock(); torch.cuda.synchronize(); lock_s = time.perf_counter() - t0
    return {"load_cases": len(cases), "iterations": it_l, "same_iterations_as_sequential": it_l == it_s,
            "sequential_s": seq_s, "lockstep_s": lock_s, "speedup": seq_s / lock_s}


def autotune_report(P, W, ctx, w, rho, f, u0, Nn):
    """The autotuner's choices for the benchmark system (check_every x smooth_sweeps of the
    two-level solve from the first timed step's warm start) and for the 8 load cases (lockstep
    group size); the bench itself runs the fixed defaults."""
    import torch
    from paper_1009_4975_gb300 import autotune as AT
    best = AT.tune_solve(ctx, rho, f, u0, check_every=(8, 16, 32), smooth_sweeps=(1, 2), repeats=3)
    cases = W.load_cases(w.dom, 8, 10)
    F = torch.zeros((len(cases), 3 * Nn), dtype=torch.float64, device=rho.device)
    for r, (nd, comp, val) in enumerate(cases):
        fr = torch.zeros(3 * Nn, dtype=torch.float64, device=rho.device)
        P.tm_build_rhs(ctx, nd, comp, val, fr)
        F[r] = fr
    bm = AT.tune_multi(ctx, rho, F, groups=(8, 4, 2), repeats=1, precond=P.TM_PRECOND_TWOLEVEL,
                       smooth_sweeps=best["smooth_sweeps"], check_every=best["check_every"])
    return {"solve": best, "multi_load": bm}


def adaptation_timing(P, ctx, rho, d, Ne, dev):
    """Adaptation step on the benchmark mesh after the timed region (not part of a step): marks
    and both sweeps on the device (CUDA events), the new leaf set on the host, and Eq. 10 between
    the two designs."""
    import torch
    r_amr = 2.0 * d.h0 / (1 << d.L)
    mk = torch.empty(Ne, dtype=torch.int8, device=dev)
    P.tm_amr_mark(ctx, rho, 0.5, r_amr, mk)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    reps = 5
    for _ in range(reps):
        P.tm_amr_mark(ctx, rho, 0.5, r_amr, mk)
    e1.record()
    torch.cuda.synchronize()
    mark_ms = e0.elapsed_time(e1) / reps
    counts = torch.bincount((mk.to(torch.int64) + 1), minlength=3).tolist()
    t0 = time.perf_counter()
    leaves, rho2 = P.tm_amr_adapt(ctx, mk, rho)
    adapt_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    dd = P.tm_design_difference(ctx, rho, leaves, rho2)
    dd_s = time.perf_counter() - t0
    return {"rho_solid": 0.5, "r_amr": r_amr, "marks": {"derefine": counts[0], "keep": counts[1],
            "refine": counts[2]}, "mark_and_sweeps_ms": mark_ms, "adapt_host_s": adapt_s,
            "new_elements": int(leaves.shape[0]), "design_difference": dd, "design_difference_s": dd_s}


def adaptive_report(P, W, w, solver, iters, every):
    """The benchmark's optimisation loop with dynamic adaptation (paper Fig. 1, Sec. 4): `iters` OC
    iterations (volume fraction 0.2) from the benchmark design, a refinement/derefinement every
    `every` iterations (marks with rho_s = 0.5, r_AMR = 2 h_min), the displacement transferred to
    each new mesh on the device as the next warm start.  Two library contexts alternate, so the old
    mesh stays resident while the new one is built.  Not part of a timed step."""
    import numpy as np
    import torch
    d = w.dom
    r_amr = 2.0 * d.h_min
    dev = torch.device("cuda", torch.cuda.current_device())

    def build(leaves):
        c = P.tm_create(dev.index, stream=torch.cuda.current_stream())
        t0 = time.perf_counter()
        info = P.tm_mesh_upload(c, d.nx, d.ny, d.nz, d.L, d.h0, leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu,
                                w.penal)
        up = time.perf_counter() - t0
        f = torch.zeros(3 * info["Nn"], dtype=torch.float64, device=dev)
        P.tm_build_rhs(c, w.load_nodes, w.load_comp, w.load_val, f)
        return c, f, info, up, P.tm_mesh_tables(c)

    wall0 = time.perf_counter()
    ctx, f, info, _, tabs = build(w.leaves)
    leaves = np.asarray(w.leaves)
    rho = torch.as_tensor(w.rho[tabs["perm"]], device=dev)
    u = torch.zeros_like(f)
    steps, remeshes = [], []
    for it in range(iters):
        st = P.tm_pcg_solve(ctx, rho, f, u, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED, **solver)
        uf = torch.zeros_like(f)
        P.tm_expand(ctx, u, uf)
        dc = torch.zeros_like(rho)
        comp = P.tm_sensitivity(ctx, rho, uf, dc)
        dch = torch.zeros_like(rho)
        P.tm_filter(ctx, rho, dc, w.r_min, 0, dch)
        new = torch.zeros_like(rho)
        chg = P.tm_oc_update(ctx, rho, dch, 0.2, 0.2, 0.5, w.rho_min, new)
        steps.append({"it": it, "elements": info["Ne"], "unknowns": info["n_free"], "iterations": st["iterations"],
                      "solve_ms": 1e3 * st["seconds"], "compliance": comp, "change": chg})
        rho = new
        if it % every != every - 1 or it == iters - 1:
            continue
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mk = torch.empty(info["Ne"], dtype=torch.int8, device=dev)
        P.tm_amr_mark(ctx, rho, 0.5, r_amr, mk)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        new_leaves, new_rho = P.tm_amr_adapt(ctx, mk, rho)
        t2 = time.perf_counter()
        ctx2, f2, info2, up, tabs2 = build(new_leaves)
        t3 = time.perf_counter()
        pts = torch.as_tensor(tabs2["node_xyz"], device=dev)
        u2 = torch.zeros(3 * info2["Nn"], dtype=torch.float64, device=dev)
        P.tm_transfer_displacement(ctx, uf, pts, u2)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        rho2 = torch.as_tensor(new_rho[tabs2["perm"]], device=dev)
        dd = P.tm_design_difference(ctx2, rho2, leaves[tabs["perm"]], rho.cpu().numpy())
        remeshes.append({"after_it": it, "elements_before": info["Ne"], "elements_after": info2["Ne"],
                         "marks_ms": 1e3 * (t1 - t0), "adapt_host_s": t2 - t1, "upload_s": up,
                         "transfer_ms": 1e3 * (t4 - t3), "design_difference": dd, "total_s": t4 - t0})
        P.tm_destroy(ctx)
        ctx, f, info, u, rho, tabs, leaves = ctx2, f2, info2, u2, rho2, tabs2, np.asarray(new_leaves)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    P.tm_destroy(ctx)
    return {"iterations": iters, "remesh_every": every, "remeshes": len(remeshes), "wall_s": wall,
            "solve_s": sum(x["solve_ms"] for x in steps) / 1e3, "remesh_s": sum(r["total_s"] for r in remeshes),
            "cg_iterations": sum(x["iterations"] for x in steps), "final_compliance": steps[-1]["compliance"],
            "elements_final": steps[-1]["elements"], "steps": steps, "remesh": remeshes}


def run_profile_apply(args):
    """Profiling workload for ncu: upload the benchmark mesh and run K FP32 operator applications."""
    import torch
    import paper_1009_4975_gb300 as P
    from paper_1009_4975_gb300 import build
    import workloads as W
    build.build()
    w = W.config2()
    d = w.dom
    ctx = P.tm_create(0, stream=torch.cuda.current_stream())
    info = P.tm_mesh_upload(ctx, d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu,
                            w.penal)
    perm = P.tm_mesh_tables(ctx)["perm"]
    rho = torch.as_tensor(w.rho[perm], device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(7)
    dt = torch.float64 if args.profile_prec == 64 else torch.float32
    x = torch.randn(3 * info["Nn"], dtype=dt, device="cuda", generator=gen)
    y = torch.zeros_like(x)
    apply = P.tm_apply_K if args.profile_prec == 64 else P.tm_apply_K_f32
    for _ in range(args.profile_apply):
        apply(ctx, rho, x, y)
    torch.cuda.synchronize()
    print(json.dumps({"profile_apply": args.profile_apply, "precision": args.profile_prec, "elements": info["Ne"]}),
          flush=True)


def _sample_workload(w=None):
    """Bounded sample of the benchmark mesh: its leaves inside the first two base-cell layers at
    the clamped face, as a mesh of its own (domain 2 x 24 x 24 base cells, same levels)."""
    import workloads as W
    w = W.config2() if w is None else w
    d = w.dom
    s = 1 << d.L
    keep = w.leaves[:, 0] < 2 * s
    dom = W.Domain(2, d.ny, d.nz, d.L, d.h0)
    ln, lc, lv = W.load_at(dom, 2 * d.h0, 0.5, 0.5)
    return W.Workload(w.name + "_first2layers", dom, w.leaves[keep], w.rho[keep], ln, lc, lv)


def _cpu_sample(full=None):
    """The oracle's reduced system on the bounded sample of the benchmark workload."""
    from oracle import fem as F
    from oracle import mesh as M
    w = _sample_workload(full)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    A, f, C = F.reduced_system(m, w.rho[m.perm], w.load_nodes, w.load_comp, w.load_val, w.E0, w.Emin, w.nu,
                               w.penal)
    return m, A, f


def _cpu_run(args, m, A, f):
    """The oracle's C/OpenMP Jacobi-PCG (all host threads) on the sample, from zero to the bench's
    tolerance."""
    from oracle import cpcg
    n = A.shape[0]
    u, it, rr, sec = cpcg.jacobi_pcg(A, f, rtol=1e-8, max_iter=args.cpu_iters)
    return {"value": n * it / sec / 1e9, "unit": UNIT, "cores": cpcg.threads(), "kind": "oracle",
            "sample": f"FP64 Jacobi-PCG (C, OpenMP CSR SpMV, {cpcg.threads()} threads; nproc {os.cpu_count()}) "
                      f"from zero to rel. residual {rr:.2e} in {it} iterations on the benchmark mesh's leaves in "
                      f"the first 2 base-cell layers at the clamped face: {m.Ne} elements, {n} unknowns",
            "seconds": sec, "time_to_tolerance_s": sec if rr <= 1e-8 else None, "iterations": it}


def cpu_baseline(args, full=None):
    return _cpu_run(args, *_cpu_sample(full))


def run_reference(args):
    """The oracle as it stands, on the host cores: W untimed and K timed runs of its Jacobi-PCG on
    the bounded sample (each run a fixed number of iterations)."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    sample = _cpu_sample()
    for _ in range(args.warmup):
        _cpu_run(args, *sample)
    t0 = time.perf_counter()
    vals = []
    cb = None
    for _ in range(max(args.steps, 1)):
        cb = _cpu_run(args, *sample)
        vals.append(cb["value"])
    wall = time.perf_counter() - t0
    value = sum(vals) / len(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded octree truss cantilever)",
            "impl": "reference", "config": {"workload": "cantilever_48x24x24_L3_truss (bounded sample)"},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-iters", type=int, default=60000,
                    help="iteration cap of the FP64 PCG comparison solve (same system as the first timed step)")
    ap.add_argument("--cpu-iters", type=int, default=100000,
                    help="iteration cap of the CPU baseline (the oracle's PCG runs to 1e-8)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="skip the batched-solve report (16 independent designs)")
    ap.add_argument("--no-reports", dest="reports", action="store_false",
                    help="skip the precision, batch and adaptation reports (profiling runs)")
    ap.add_argument("--precond", default="twolevel", choices=["twolevel", "jacobi"],
                    help="preconditioner of the chosen (mixed) solver")
    ap.add_argument("--nu", type=int, default=2, help="two-level: l1-Jacobi sweeps before and after the coarse step")
    ap.add_argument("--check-every", type=int, default=8,
                    help="CG iterations per CUDA-graph batch (iterations enqueued past convergence return at once)")
    ap.add_argument("--adaptive-iters", type=int, default=60,
                    help="report: OC iterations of the adaptive loop with remeshing (0: skip)")
    ap.add_argument("--remesh-every", type=int, default=5, help="report: OC iterations between remeshes")
    ap.add_argument("--no-graphs", action="store_true",
                    help="plain kernel launches instead of CUDA-graph batches (for launch-list profiling)")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="profiling workload: K operator applications on the benchmark mesh, no timing")
    ap.add_argument("--profile-prec", type=int, default=32, choices=[32, 64],
                    help="profiling workload: FP32 (tm_apply_K_f32) or FP64 (tm_apply_K) operator")
    args = ap.parse_args()
    if args.profile_apply > 0:
        run_profile_apply(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
