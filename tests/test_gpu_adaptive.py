"""The adaptive optimisation loop on the GPU (paper Fig. 1 and Sec. 4): OC iterations with a
mesh refinement/derefinement every 5 iterations, the displacement carried to each new mesh as the
warm start of the next solve.

Every step runs through the C ABI on two library contexts that alternate (the old mesh stays
resident while the new one is built).  At each remesh the test checks against the oracle:
* the marks after both sweeps and the new leaf set with its densities, bit for bit;
* the design difference of Eq. 10 between the designs before and after the remesh;
* the device displacement transfer against the oracle's evaluation of the old field at the new
  nodes (the same trilinear interpolation in FP64: 1e-14 of the field's scale);
and after it, that the warm-started solve on the new mesh reaches a residual of 1e-8 in the
oracle's A of that mesh in fewer iterations than the same solve from zero.
"""
import numpy as np
import pytest

import workloads as W
from oracle import amr as A
from oracle import fem as F
from oracle import mesh as M
from tests.gpu_common import tm

pytestmark = pytest.mark.gpu

ITERS, EVERY, VOLFRAC = 10, 5, 0.3


def _context(w, leaves):
    import torch
    P = tm()
    d = w.dom
    c = P.tm_create(0, stream=torch.cuda.current_stream())
    info = P.tm_mesh_upload(c, d.nx, d.ny, d.nz, d.L, d.h0, leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu, w.penal)
    f = torch.zeros(3 * info["Nn"], dtype=torch.float64, device="cuda")
    P.tm_build_rhs(c, w.load_nodes, w.load_comp, w.load_val, f)
    return c, f


@pytest.mark.parametrize("precond", [0, 1])
def test_adaptive_loop_with_remeshing_and_warm_starts(precond):
    import torch
    P = tm()
    w = W.config1b()
    d = w.dom
    r_amr = 2.0 * d.h_min
    leaves = np.asarray(w.leaves, np.int64)
    ctx, f = _context(w, leaves)
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, leaves, dirichlet_faces=w.dirichlet_faces)
    rho = torch.as_tensor(w.rho[m.perm], device="cuda")
    u = torch.zeros_like(f)
    remeshes = 0
    try:
        for it in range(ITERS):
            st = P.tm_pcg_solve(ctx, rho, f, u, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                                precond=precond)
            uf = torch.zeros_like(f)
            P.tm_expand(ctx, u, uf)
            dc = torch.zeros_like(rho)
            P.tm_sensitivity(ctx, rho, uf, dc)
            dch = torch.zeros_like(rho)
            P.tm_filter(ctx, rho, dc, w.r_min, 0, dch)
            new = torch.zeros_like(rho)
            P.tm_oc_update(ctx, rho, dch, VOLFRAC, 0.2, 0.5, w.rho_min, new)
            rho = new
            if it % EVERY != EVERY - 1:
                continue
            # ---- remesh: marks and the new leaf set on the old mesh
            rho_h = rho.cpu().numpy()
            mk = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
            P.tm_amr_mark(ctx, rho, 0.5, r_amr, mk)
            want = A.final_marks(m, rho_h, 0.5, r_amr)
            np.testing.assert_array_equal(mk.cpu().numpy(), want)
            new_leaves, new_rho = P.tm_amr_adapt(ctx, mk, rho)
            wl, wr = A.adapt(m, want, rho_h)
            np.testing.assert_array_equal(new_leaves, wl)
            assert new_rho.tobytes() == wr.tobytes()
            assert not np.array_equal(np.sort(new_leaves, axis=0), np.sort(m.leaves, axis=0))
            # ---- the new mesh in the other context; the old field at its nodes
            ctx2, f2 = _context(w, new_leaves)
            m2 = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, new_leaves, dirichlet_faces=w.dirichlet_faces)
            rho2 = torch.as_tensor(new_rho[m2.perm], device="cuda")
            dd = P.tm_design_difference(ctx2, rho2, m.leaves, rho_h)
            dd_o = A.design_difference(d.nx, d.ny, d.nz, d.L, m2.leaves, new_rho[m2.perm], m.leaves, rho_h)
            assert abs(dd - dd_o) <= 1e-12 * max(1.0, abs(dd_o))
            pts = torch.as_tensor(P.tm_mesh_tables(ctx2)["node_xyz"], device="cuda")
            u2 = torch.zeros(3 * m2.Nn, dtype=torch.float64, device="cuda")
            P.tm_transfer_displacement(ctx, uf, pts, u2)
            ut = A.transfer_field(m, uf.cpu().numpy(), m2.nodes).ravel()
            scale = np.abs(ut).max()
            assert np.abs(u2.cpu().numpy() - ut).max() <= 1e-14 * scale
            P.tm_destroy(ctx)
            ctx, f, m, rho, u = ctx2, f2, m2, rho2, u2
            remeshes += 1
            # ---- the warm-started solve on the new mesh, judged in the oracle's A
            A2, fv, _ = F.reduced_system(m, rho.cpu().numpy(), w.load_nodes, w.load_comp, w.load_val, w.E0,
                                         w.Emin, w.nu, w.penal)
            uw = u.clone()
            stw = P.tm_pcg_solve(ctx, rho, f, uw, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                                 precond=precond)
            ufree = F.from_full_layout(m, uw.cpu().numpy())
            assert np.linalg.norm(fv - A2 @ ufree) <= 1.0001e-8 * np.linalg.norm(fv)
            u0 = torch.zeros_like(f)
            st0 = P.tm_pcg_solve(ctx, rho, f, u0, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                                 precond=precond)
            assert stw["iterations"] < st0["iterations"], (stw["iterations"], st0["iterations"])
        assert remeshes == ITERS // EVERY
    finally:
        P.tm_destroy(ctx)


def test_transfer_rejects_points_outside_the_box():
    import torch
    P = tm()
    w = W.config1()
    ctx, f = _context(w, w.leaves)
    try:
        uf = torch.zeros_like(f)
        fx = w.dom.nx << w.dom.L
        pts = torch.tensor([[0, 0, 0], [fx + 1, 0, 0]], dtype=torch.int32, device="cuda")
        out = torch.zeros(6, dtype=torch.float64, device="cuda")
        with pytest.raises(P.TmError) as e:
            P.tm_transfer_displacement(ctx, uf, pts, out)
        assert e.value.code == P.TM_EINVAL
    finally:
        P.tm_destroy(ctx)
