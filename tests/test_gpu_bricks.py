"""The operator's brick pass on a mesh where it meets every case it handles: aligned 4x4x4
bricks of equal-level elements next to finer and coarser elements, so that some bricks have
hanging lattice nodes on faces and edges (interpolated from, and folded into, lattice nodes one
step away), bricks with Dirichlet lattice nodes on the clamped face, and record-driven blocks
filled from the elements between bricks.

* The FP64 and FP32 operators equal the oracle's assembled C^T K C x within 256 u (|A| |x|)_i
  (the reordered-sum bound of `test_gpu_parity.py`).
* Applying the operator to several vectors at once gives each vector's single application bit
  for bit (the multi-vector kernel runs the same brick and block code vector after vector).
* The mixed two-level solve reaches the parity criterion in the oracle's A.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import U32, U64, Case, ctx, tm

pytestmark = pytest.mark.gpu


def _truss_case():
    w = W.small_truss(seed=4, base=(8, 4, 4), L=2)
    return w, Case(w)


@pytest.fixture(scope="module")
def bricked():
    w, c = _truss_case()
    d = w.dom
    ops = tm().tm_tables_operator(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces)
    c.ops = ops
    c.info = c.upload()
    return c


def test_the_mesh_exercises_every_brick_case(bricked):
    ops = bricked.ops
    nb = ops["info"]["n_bricks"]
    hax, node = ops["brick_hax"], ops["brick_node"]
    assert nb > 0 and ops["info"]["n_blocks"] > 0
    assert bricked.info["n_bricks"] == nb
    # bricks with hanging lattice nodes: edge-hanging (one axis) and face-hanging (two axes)
    masks = set(int(v) for v in hax[hax != 0].ravel())
    assert masks & {1, 2, 4} and masks & {3, 5, 6}
    # bricks with Dirichlet lattice nodes
    assert np.any(node < 0)
    # bricks hold most of the elements
    assert 64 * nb > 0.5 * bricked.m.Ne


@pytest.mark.parametrize("prec", [64, 32])
def test_operator_matches_the_assembled_matrix(bricked, prec):
    import torch
    P = tm()
    c = bricked
    rho = c.t(c.rho)
    x = np.random.default_rng(21).standard_normal(c.A.shape[0])
    if prec == 64:
        y = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device=c.dev)
        P.tm_apply_K(ctx(), rho, c.t(c.full(x)), y)
        u, xin = U64, x
    else:
        xin = x.astype(np.float32).astype(np.float64)          # the FP32 input, exactly
        y = torch.zeros(3 * c.m.Nn, dtype=torch.float32, device=c.dev)
        P.tm_apply_K_f32(ctx(), rho, c.t(c.full(xin), torch.float32), y)
        u = U32
    got = c.free(y.double().cpu().numpy())
    err = np.abs(got - c.A @ xin)
    assert np.all(err <= 256 * u * (abs(c.A) @ np.abs(xin)))


def test_multi_vector_operator_is_bitwise_the_single_one(bricked):
    import torch
    P = tm()
    c = bricked
    rho = c.t(c.rho)
    n3 = 3 * c.m.Nn
    X = torch.as_tensor(np.random.default_rng(22).standard_normal((3, n3)), dtype=torch.float32, device=c.dev)
    X *= torch.as_tensor(np.repeat(c.m.dirichlet == 0, 3), dtype=torch.float32, device=c.dev)
    Y = torch.zeros_like(X)
    P.tm_apply_K_f32_multi(ctx(), rho, X, Y)
    for r in range(3):
        y = torch.zeros(n3, dtype=torch.float32, device=c.dev)
        P.tm_apply_K_f32(ctx(), rho, X[r].contiguous(), y)
        assert torch.equal(y, Y[r]), r


def test_two_level_mixed_solve_reaches_the_parity_criterion(bricked):
    import torch
    P = tm()
    c = bricked
    rho = c.t(c.rho)
    f = c.t(c.full(c.f))
    u = torch.zeros_like(f)
    st = P.tm_pcg_solve(ctx(), rho, f, u, rtol=1e-8, max_iter=100000, precision=P.TM_PREC_MIXED,
                        precond=P.TM_PRECOND_TWOLEVEL)
    assert st["status"] == 0
    uf = c.free(u.cpu().numpy())
    assert np.linalg.norm(c.f - c.A @ uf) / np.linalg.norm(c.f) <= 1e-8 * (1 + 1e-3)
