"""Autotuner of the solver's launch parameters for one uploaded mesh.

The tuned parameters are the ones the library takes per call rather than per build:
* ``check_every``: CG iterations per CUDA-graph batch (a larger batch saves host round trips;
  iterations enqueued past a stopping point return at once but still cost a launch each);
* ``smooth_sweeps``: l1-Jacobi sweeps per level of the two-level V-cycle (fewer iterations
  against a costlier iteration);
* for several load cases, the lockstep group size (all cases in one group, or groups of 4, 2
  or 1 solved one after another).

Each candidate is timed with the library's own solve on the caller's system (a warm-up solve
first, then the median of `repeats` timed solves from the same start), and the fastest is kept in
a cache keyed by the mesh's sizes.  Only library calls run here; torch holds the buffers.
"""
from __future__ import annotations

import time

from . import tm as T

_cache: dict = {}


def _key(ctx, kind):
    i = ctx.info
    return (kind, i["Ne"], i["Nn"], i["n_hanging"], i["n_blocks"])


def _timed(fn, repeats):
    import torch
    fn()
    ts = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    ts.sort()
    return ts[len(ts) // 2]


def tune_solve(ctx, rho, f, u0, check_every=(8, 16, 32), smooth_sweeps=(1, 2), repeats=3, refresh=False):
    """Fastest (check_every, smooth_sweeps) of the two-level mixed solve of rho, f from u0 (u0 is
    not modified).  Returns {"check_every", "smooth_sweeps", "seconds", "table"}."""
    key = _key(ctx, "solve")
    if key in _cache and not refresh:
        return _cache[key]
    table = []
    for ce in check_every:
        for nu in smooth_sweeps:
            def run(ce=ce, nu=nu):
                u = u0.clone()
                T.tm_pcg_solve(ctx, rho, f, u, rtol=1e-8, max_iter=200000, precision=T.TM_PREC_MIXED,
                               precond=T.TM_PRECOND_TWOLEVEL, smooth_sweeps=nu, check_every=ce)
            table.append({"check_every": ce, "smooth_sweeps": nu, "seconds": _timed(run, repeats)})
    best = min(table, key=lambda r: (r["seconds"], r["check_every"], r["smooth_sweeps"]))
    _cache[key] = dict(best, table=table)
    return _cache[key]


def tune_multi(ctx, rho, F, groups=(8, 4, 2, 1), repeats=2, refresh=False, **solver):
    """Fastest lockstep group size for the load cases in the rows of F (nrhs, 3 Nn), each group a
    tm_pcg_solve_multi call and the groups solved one after another.  Returns {"group",
    "seconds", "table"}."""
    import torch
    nr = int(F.shape[0])
    key = _key(ctx, ("multi", nr))
    if key in _cache and not refresh:
        return _cache[key]
    table = []
    for gsz in groups:
        if gsz > nr or gsz > 8:
            continue

        def run(gsz=gsz):
            U = torch.zeros_like(F)
            for a in range(0, nr, gsz):
                b = min(nr, a + gsz)
                T.tm_pcg_solve_multi(ctx, rho, F[a:b].contiguous(), U[a:b].contiguous(), rtol=1e-8,
                                     max_iter=200000, **solver)
        table.append({"group": gsz, "seconds": _timed(run, repeats)})
    best = min(table, key=lambda r: (r["seconds"], -r["group"]))
    _cache[key] = dict(best, table=table)
    return _cache[key]
