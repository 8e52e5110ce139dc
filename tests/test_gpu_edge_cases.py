"""Degenerate and boundary cases of the GPU path against the oracle: a one-element mesh,
uniform meshes without hanging nodes (coarsest and finest level), other residual-replacement
ratios of the mixed solver, and adaptation of all-void and all-solid designs."""
import numpy as np
import pytest

import workloads as W
from oracle import amr as A
from oracle import mesh as M
from tests.gpu_common import U64, Case, ctx, tm

pytestmark = pytest.mark.gpu


def _workload(dom, leaves, load_node, seed=0):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 1.0, len(leaves))
    return W.Workload("edge", dom, np.asarray(leaves, np.int64), rho, np.array([load_node], np.int64),
                      np.array([2], np.int64), np.array([-1.0]))


def _check_operator_and_solves(c):
    import torch
    P = tm()
    c.info = c.upload()
    rho = c.t(c.rho)
    # FP64 operator against the assembled reduced matrix
    rng = np.random.default_rng(3)
    x = rng.standard_normal(c.A.shape[0])
    y = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device=c.dev)
    P.tm_apply_K(ctx(), rho, c.t(c.full(x)), y)
    torch.cuda.synchronize()
    err = np.abs(c.free(y.cpu().numpy()) - c.A @ x)
    assert np.all(err <= 256 * U64 * (abs(c.A) @ np.abs(x)))
    # both solvers reach the parity criterion in the oracle's A
    f = torch.zeros_like(y)
    P.tm_build_rhs(ctx(), c.w.load_nodes, c.w.load_comp, c.w.load_val, f)
    for prec in (P.TM_PREC_FP64, P.TM_PREC_MIXED):
        u = torch.zeros_like(f)
        st = P.tm_pcg_solve(ctx(), rho, f, u, rtol=1e-8, max_iter=100000, precision=prec)
        assert st["status"] == 0
        uf = c.free(u.cpu().numpy())
        assert np.linalg.norm(c.f - c.A @ uf) / np.linalg.norm(c.f) <= 1e-8 * (1 + 1e-3)


def test_one_element_mesh():
    dom = W.Domain(1, 1, 1, 0, 1.0)
    c = Case(_workload(dom, [[0, 0, 0, 0]], [1, 1, 1]))
    assert c.m.Ne == 1 and c.m.Nn == 8 and not c.m.hanging
    _check_operator_and_solves(c)


@pytest.mark.parametrize("level", [0, 2])
def test_uniform_meshes_without_hanging_nodes(level):
    dom = W.Domain(6, 3, 3, 2, 2.0 / 6)
    leaves = W.uniform_leaves(dom)
    for _ in range(level):
        leaves = W.refine(dom, leaves, np.ones(len(leaves), bool))
    c = Case(_workload(dom, leaves, [24, 4, 4], seed=level))
    assert not c.m.hanging and c.m.Ne == 54 * 8 ** level
    _check_operator_and_solves(c)


@pytest.mark.parametrize("ratio", [0.5, 0.01])
def test_mixed_solver_replacement_ratios(ratio):
    import torch
    P = tm()
    c = Case(W.config1b())
    c.upload()
    f = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device=c.dev)
    P.tm_build_rhs(ctx(), c.w.load_nodes, c.w.load_comp, c.w.load_val, f)
    u = torch.zeros_like(f)
    st = P.tm_pcg_solve(ctx(), c.t(c.rho), f, u, rtol=1e-8, max_iter=100000, precision=P.TM_PREC_MIXED,
                        inner_rtol=ratio)
    assert st["status"] == 0 and st["sweeps"] >= 1
    uf = c.free(u.cpu().numpy())
    assert np.linalg.norm(c.f - c.A @ uf) / np.linalg.norm(c.f) <= 1e-8 * (1 + 1e-3)


@pytest.mark.parametrize("value", [1e-3, 1.0])
def test_adaptation_of_uniform_designs(value):
    import torch
    P = tm()
    w = W.config1b(2)
    d = w.dom
    P.tm_mesh_upload(ctx(), d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces)
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    rho = np.full(m.Ne, value)
    rho_d = torch.as_tensor(rho, device="cuda:0")
    mk = torch.empty(m.Ne, dtype=torch.int8, device="cuda:0")
    P.tm_amr_mark(ctx(), rho_d, 0.5, 1.5 * d.h_min, mk)
    got = mk.cpu().numpy()
    want = A.final_marks(m, rho, 0.5, 1.5 * d.h_min)
    np.testing.assert_array_equal(got, want)
    if value == 1.0:          # all solid: everything below the finest level refines
        assert np.array_equal(got == 1, m.leaves[:, 3] < d.L)
    else:                     # all void: no element refines
        assert not (got == 1).any() and (got == -1).any()
    gl, gr = P.tm_amr_adapt(ctx(), mk, rho_d)
    wl, wr = A.adapt(m, want, rho)
    np.testing.assert_array_equal(gl, wl)
    assert gr.tobytes() == wr.tobytes()
    assert P.tm_design_difference(ctx(), rho_d, gl, gr) == 0.0
