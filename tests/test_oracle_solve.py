"""Pins for the oracle's solvers (paper Sec. 5) against dense factorisation and beam theory."""
import numpy as np
import pytest

import workloads as W
from oracle import fem as F
from oracle import mesh as M
from oracle import solve as S

NU = 0.3


def _system(w):
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    rho = w.rho[m.perm]
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val)
    return m, rho, A, f, C


def test_sparse_direct_matches_textbook_dense_cholesky():
    dom = W.Domain(4, 2, 2, 1, 0.5)
    w = W.random_field_mesh("tiny", dom, 7, [(0.2, 0.8)])
    w.rho = 0.2 + 0.8 * w.rho          # moderate contrast: both factorisations stay accurate
    m, rho, A, f, C = _system(w)
    assert A.shape[0] < 600
    Lm = S.dense_cholesky(A.toarray())
    ud = S.cholesky_solve(Lm, f)
    us = S.direct(A, f)
    assert np.abs(ud - us).max() <= 1e-10 * np.abs(us).max()
    assert S.relative_residual(A, us, f) < 1e-12


def test_jacobi_pcg_reaches_direct_solution():
    w = W.config1()
    m, rho, A, f, C = _system(w)
    u = S.direct(A, f)
    up, it, rr, _ = S.jacobi_pcg(A, f, rtol=1e-12)
    assert rr <= 1e-12
    assert S.relative_residual(A, up, f) < 1e-11
    # energy-norm error of CG is what the residual controls; compliance converges fast
    assert abs(f @ up - f @ u) <= 1e-9 * abs(f @ u)
    # warm start from the solution needs no iterations
    _, it0, _, _ = S.jacobi_pcg(A, f, u0=u, rtol=1e-8)
    assert it0 == 0


def _tip_deflection(k):
    dom = W.Domain(8 * k, k, k, 0, 1.0 / k)
    m = M.build_mesh(dom.nx, dom.ny, dom.nz, 0, dom.h0, W.uniform_leaves(dom))
    tip = np.nonzero(m.nodes[:, 0] == 8 * k)[0]
    yz = m.nodes[tip][:, 1:]
    wgt = np.where((yz == 0) | (yz == k), 0.5, 1.0).prod(axis=1)
    wgt = wgt / wgt.sum()          # consistent nodal loads of a uniform traction, total -1
    A, f, C = F.reduced_system(m, np.ones(m.Ne), m.nodes[tip], np.full(tip.size, 2), -wgt, Emin=0.0)
    uf = (C @ S.direct(A, f)).reshape(-1, 3)
    return -(uf[tip, 2] * wgt).sum()


def test_cantilever_tip_deflection_converges_to_timoshenko():
    """Slender 8 x 1 x 1 box, E = 1, nu = 0.3, clamped at x = 0, unit shear load on the tip:
    delta = F L^3 / (3 E I) + F L / (kappa G A) with kappa = 5/6."""
    G = 1.0 / (2 * (1 + NU))
    exact = 8.0 ** 3 / (3.0 / 12.0) + 8.0 / (5.0 / 6.0 * G)
    d = [_tip_deflection(k) for k in (2, 4, 8)]
    assert d[0] < d[1] < d[2] < exact
    assert abs(d[2] / exact - 1) < 0.025
    aitken = d[2] - (d[2] - d[1]) ** 2 / ((d[2] - d[1]) - (d[1] - d[0]))
    assert abs(aitken / exact - 1) < 0.01


def test_refined_mesh_agrees_with_uniform_mesh_on_a_linear_solution():
    """A pure tension field is represented exactly on any mesh: uniform and AMR meshes give
    the same displacements at shared nodes (AMR's premise, Sec. 1)."""
    dom = W.Domain(4, 2, 2, 1, 0.5)
    lv_uni = W.refine(dom, W.uniform_leaves(dom), np.ones(16, bool))
    lv_amr = W.refine(dom, W.uniform_leaves(dom), np.arange(16) % 3 == 0)
    out = []
    for leaves in (lv_uni, lv_amr):
        m = M.build_mesh(4, 2, 2, 1, 0.5, leaves, dirichlet_faces=0b1)
        tip = np.nonzero(m.nodes[:, 0] == 8)[0]
        yz = m.nodes[tip][:, 1:]
        # consistent nodal loads of a uniform traction on the tip face (finest unit 0.25)
        wgt = np.zeros(tip.size)
        lk = {tuple(p): i for i, p in enumerate(map(tuple, m.nodes[tip]))}
        for e in range(m.Ne):
            s = 1 << (1 - m.leaves[e, 3])
            if m.leaves[e, 0] + s != 8:
                continue
            for k in (1, 3, 5, 7):
                p = tuple(m.leaves[e, :3] + s * M.CORNER_OFFSETS[k])
                wgt[lk[p]] += (s * 0.25) ** 2 / 4.0     # physical face area / 4
        A, f, C = F.reduced_system(m, np.ones(m.Ne), m.nodes[tip], np.zeros(tip.size, int), wgt, Emin=0.0, nu=0.0)
        uf = (C @ S.direct(A, f)).reshape(-1, 3)
        out.append({tuple(p): uf[i] for i, p in enumerate(map(tuple, m.nodes))})
    common = set(out[0]) & set(out[1])
    assert len(common) > 20
    # nu = 0 and a clamped face that only has to resist x: uniaxial tension, u_x = sigma x / E
    for p in common:
        assert np.allclose(out[0][p], out[1][p], atol=1e-11)
        assert abs(out[0][p][0] - p[0] * 0.25) < 1e-11


# ---------------------------------------------------------------- two-level preconditioner
def _twolevel_case():
    import workloads as W
    from oracle import fem as F
    from oracle import mesh as M
    w = W.config1b()
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    A, f, C = F.reduced_system(m, w.rho[m.perm], w.load_nodes, w.load_comp, w.load_val)
    return m, A.tocsr(), f


def test_grid_prolongation_reproduces_linear_fields_at_free_nodes():
    from oracle import fem as F
    from oracle import learn as LR
    m, A, f = _twolevel_case()
    P = S.grid_prolongation(m, 1)
    X, Y, Z = LR.grid_shape(m, 1)
    hv = 1 << (m.L - 1)
    cx, cy, cz = np.meshgrid((np.arange(X) + 0.5) * hv, (np.arange(Y) + 0.5) * hv, (np.arange(Z) + 0.5) * hv,
                             indexing="ij")
    B = np.array([[0.5, -0.25, 1.0], [2.0, 0.75, -1.5], [-0.125, 0.3, 0.6]])
    cells = np.stack([cx, cy, cz], -1).reshape(-1, 3) @ B.T          # (ncell, 3), cell-major
    nodal = m.nodes[F.free_nodes(m)].astype(np.float64) @ B.T
    np.testing.assert_allclose(P @ cells.ravel(), nodal.ravel(), rtol=1e-12, atol=1e-12 * np.abs(nodal).max())


def test_galerkin_correction_is_exact_on_the_coarse_space():
    """If u* = P c, then P (P^T A P)^-1 P^T A u* = u* (Galerkin projection)."""
    m, A, f = _twolevel_case()
    P = S.grid_prolongation(m, 0)
    c = np.random.default_rng(3).standard_normal(P.shape[1])
    us = P @ c
    got = S.coarse_correction(A, P)(A @ us)
    assert np.abs(got - us).max() <= 1e-8 * np.abs(us).max()


def test_twolevel_preconditioner_is_spd_and_cuts_iterations():
    m, A, f = _twolevel_case()
    P = S.grid_prolongation(m, 1)
    dinv = 1.0 / A.diagonal()
    cc = S.coarse_correction(A, P)
    Minv = lambda r: dinv * r + cc(r)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    assert a @ Minv(b) == pytest.approx(b @ Minv(a), rel=1e-8)
    assert a @ Minv(a) > 0
    u2, it2, _ = S.twolevel_pcg(A, f, P, rtol=1e-8)
    u1, it1, _, _ = S.jacobi_pcg(A, f, rtol=1e-8)
    assert np.linalg.norm(f - A @ u2) <= 1.01e-8 * np.linalg.norm(f)
    ud = S.direct(A, f)
    e = u2 - ud
    assert np.sqrt(e @ (A @ e) / (ud @ (A @ ud))) <= 1e-6
    assert it2 * 3 <= it1


def test_cell_transfer_is_exact_for_linear_fields():
    X, Y, Z = 8, 4, 6
    T = S.cell_transfer(X, Y, Z)
    B = np.array([[0.5, -0.25, 1.0], [2.0, 0.75, -1.5], [-0.125, 0.3, 0.6]])
    def centres(nx, ny, nz, h):
        cx, cy, cz = np.meshgrid((np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nz) + 0.5) * h,
                                 indexing="ij")
        return np.stack([cx, cy, cz], -1).reshape(-1, 3)
    coarse = centres(X // 2, Y // 2, Z // 2, 2.0) @ B.T
    fine = centres(X, Y, Z, 1.0) @ B.T
    np.testing.assert_allclose(T @ coarse.ravel(), fine.ravel(), rtol=1e-12, atol=1e-12)


def test_vcycle_is_spd_and_keeps_most_of_the_coarse_gain():
    from oracle import learn as LR
    w = W.small_truss(seed=4, base=(8, 4, 4), L=2)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    A, f, C = F.reduced_system(m, w.rho[m.perm], w.load_nodes, w.load_comp, w.load_val)
    A = A.tocsr()
    P = S.grid_prolongation(m, 1)
    shape = LR.grid_shape(m, 1)
    V = S.VCycle((P.T @ A @ P).tocsr(), shape, nu=2)
    assert len(V.levels) == 3
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal(P.shape[1]), rng.standard_normal(P.shape[1])
    assert a @ V.apply(b) == pytest.approx(b @ V.apply(a), rel=1e-8)
    assert a @ V.apply(a) > 0
    u, it_v, _ = S.twolevel_vcycle_pcg(A, f, P, shape, nu=2)
    it_j = S.jacobi_pcg(A, f, rtol=1e-8)[1]
    assert np.linalg.norm(f - A @ u) <= 1.01e-8 * np.linalg.norm(f)
    assert 4 * it_v <= it_j
