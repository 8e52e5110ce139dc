"""Concurrent independent solves (tm_pcg_solve_batch): each solve of the batch gives the
same u, bit for bit, and the same iteration count as the same solve run alone, and meets
the solve parity criterion (residual in the oracle's A)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import Case, tm

pytestmark = pytest.mark.gpu


def _setup(P, w, stream):
    import torch
    c = Case(w)
    d = w.dom
    ctx = P.tm_create(0, stream=stream)
    P.tm_mesh_upload(ctx, d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu, w.penal)
    f = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device="cuda:0")
    with torch.cuda.stream(stream):
        P.tm_build_rhs(ctx, w.load_nodes, w.load_comp, w.load_val, f)
    return c, ctx, c.t(c.rho), f


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_individual_solves(precision):
    import torch
    P = tm()
    works = [W.config1(), W.config1b(), W.config1b(3), W.small_truss(seed=4, base=(8, 4, 4), L=2)]
    streams = [torch.cuda.Stream() for _ in works]
    items = [_setup(P, w, s) for w, s in zip(works, streams)]
    torch.cuda.synchronize()
    alone = []
    for c, ctx, rho, f in items:
        u = torch.zeros_like(f)
        st = P.tm_pcg_solve(ctx, rho, f, u, rtol=1e-8, max_iter=200000, precision=precision)
        torch.cuda.synchronize()
        alone.append((u.cpu().numpy(), st["iterations"]))
    us = [torch.zeros_like(f) for _, _, _, f in items]
    torch.cuda.synchronize()
    stats = P.tm_pcg_solve_batch([it[1] for it in items], [it[2] for it in items], [it[3] for it in items], us,
                                 rtol=1e-8, max_iter=200000, precision=precision)
    torch.cuda.synchronize()
    for (c, ctx, rho, f), u, st, (ua, ita) in zip(items, us, stats, alone):
        assert st["status"] == 0
        assert st["iterations"] == ita
        got = u.cpu().numpy()
        assert got.tobytes() == ua.tobytes()
        uf = c.free(got)
        assert np.linalg.norm(c.f - c.A @ uf) / np.linalg.norm(c.f) <= 1e-8 * (1 + 1e-3)
    for _, ctx, _, _ in items:
        P.tm_destroy(ctx)


def test_batch_rejects_a_repeated_context():
    import torch
    P = tm()
    s = torch.cuda.Stream()
    c, ctx, rho, f = _setup(P, W.config1(), s)
    torch.cuda.synchronize()
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    with pytest.raises(P.TmError):
        P.tm_pcg_solve_batch([ctx, ctx], [rho, rho], [f, f], [u1, u2])
    P.tm_destroy(ctx)
