"""Pins for the oracle of the two-level preconditioner (oracle/coarse.py).

Each pin checks the oracle against something fixed outside it: exact interpolation of linear
fields, the hanging-node constraints of the fine mesh, a direct Gauss quadrature of the coarse
basis against the piecewise-constant Young's modulus, the spectrum of the smoother, the symmetry
and definiteness of the cycle, and the direct solution of the system.
"""
import numpy as np
import pytest

import workloads as W
from oracle import coarse as CO
from oracle import fem as F
from oracle import mesh as M
from oracle import solve as S

B_LIN = np.array([[0.5, -0.25, 1.0], [2.0, 0.75, -1.5], [-0.125, 0.3, 0.6]])
A_LIN = np.array([0.3, -0.7, 0.2])


def _mesh(w, faces=None):
    d = w.dom
    faces = w.dirichlet_faces if faces is None else faces
    return M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=faces)


def _system(w):
    m = _mesh(w)
    rho = w.rho[m.perm]
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val)
    return m, rho, A.tocsr(), f, C


def test_level_shapes_follow_the_halving_rule():
    m = _mesh(W.config1b())
    assert CO.level_shapes(m) == [(8, 4, 4), (4, 2, 2)]
    dom = W.Domain(48, 24, 24, 0, 1.0 / 24)
    fake = M.Mesh(48, 24, 24, 0, 1.0 / 24, np.zeros((1, 4), np.int64), np.zeros(1, np.int64),
                  np.zeros((1, 3), np.int64), np.zeros((1, 8), np.int64), {}, np.zeros(1, bool))
    assert CO.level_shapes(fake) == [(48, 24, 24), (24, 12, 12), (12, 6, 6), (6, 3, 3)]
    assert dom.nx == 48
    odd = M.Mesh(18, 9, 9, 0, 1.0, fake.leaves, fake.perm, fake.nodes, fake.conn, {}, fake.dirichlet)
    assert CO.level_shapes(odd) == [(18, 9, 9), (9, 5, 5), (5, 3, 3)]
    # an odd count on an axis with a clamped upper face ends the hierarchy
    assert CO.level_shapes(odd, dirichlet_faces=1 | 8) == [(18, 9, 9)]


def test_fine_prolongation_reproduces_linear_fields_at_free_nodes():
    m = _mesh(W.config1b(), faces=0)           # no clamped face: every lattice node is free
    P0 = CO.fine_prolongation(m, dirichlet_faces=0)
    S_ = 1 << m.L
    lat = CO.lattice_nodes((m.nx, m.ny, m.nz)) * S_          # lattice nodes in finest units
    coarse = A_LIN + lat.astype(np.float64) @ B_LIN.T
    fine = A_LIN + m.nodes[F.free_nodes(m)].astype(np.float64) @ B_LIN.T
    np.testing.assert_allclose(P0 @ coarse.ravel(), fine.ravel(), rtol=1e-13, atol=1e-13 * np.abs(fine).max())


def test_coarse_space_lies_in_the_finite_element_space():
    """C (P0 v) -- the fine field with hanging values interpolated from their masters (Eq. 6) --
    equals the trilinear interpolant of v at every mesh node, hanging ones included; nodes on
    the clamped face get 0 from both sides."""
    w = W.config1b()
    m = _mesh(w)
    P0 = CO.fine_prolongation(m)
    C = F.constraint_matrix(m)
    X, Y, Z = m.nx, m.ny, m.nz
    free = CO.lattice_free((X, Y, Z), 1)
    v = np.random.default_rng(5).standard_normal(3 * free.size)
    vall = np.zeros((X + 1) * (Y + 1) * (Z + 1) * 3)
    vall.reshape(-1, 3)[free] = v.reshape(-1, 3)
    S_ = 1 << m.L
    p = m.nodes.astype(np.int64)
    cell = np.minimum(p // S_, np.array([X - 1, Y - 1, Z - 1]))
    t = (p - cell * S_) / S_
    want = np.zeros((m.Nn, 3))
    for q in range(8):
        a, b, c = q & 1, (q >> 1) & 1, q >> 2
        wq = (t[:, 0] if a else 1 - t[:, 0]) * (t[:, 1] if b else 1 - t[:, 1]) * (t[:, 2] if c else 1 - t[:, 2])
        J = (cell[:, 0] + a) + (X + 1) * ((cell[:, 1] + b) + (Y + 1) * (cell[:, 2] + c))
        want += wq[:, None] * vall.reshape(-1, 3)[J]
    got = (C @ (P0 @ v)).reshape(-1, 3)
    assert len(m.hanging) > 0
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("level", [0, 1])
def test_galerkin_operator_equals_quadrature_of_the_cell_basis(level):
    w = W.config1b()
    m, rho, A, f, C = _system(w)
    H = CO.Hierarchy(m, A)
    assert H.levels == 2
    K = CO.quadrature_cell_matrices(m, rho, level, w.E0, w.Emin, w.nu, w.penal)
    Aq = CO.assemble_cells(CO.level_shapes(m)[level], K)
    diff = abs(H.A[level] - Aq).max()
    assert diff <= 1e-12 * abs(Aq).max()


def test_cell_quadrature_of_a_single_leaf_cell_is_its_element_matrix():
    """A base cell that is one leaf of side h0: K_C = E h0 K0 (the fine element matrix)."""
    w = W.config1()
    m = _mesh(w)
    rho = w.rho[m.perm]
    K = CO.quadrature_cell_matrices(m, rho, 0, w.E0, w.Emin, w.nu, w.penal)
    K0 = F.reference_stiffness(w.nu)
    E = F.young(rho, w.E0, w.Emin, w.penal)
    one = np.nonzero(m.leaves[:, 3] == 0)[0]
    assert one.size > 0
    for e in one[:5]:
        ix, iy, iz, _ = (int(v) for v in m.leaves[e] // (1 << m.L))
        ci = ix + m.nx * (iy + m.ny * iz)
        np.testing.assert_allclose(K[ci], E[e] * m.h0 * K0, rtol=1e-12, atol=1e-12 * E[e] * np.abs(K0).max())


def test_level_prolongation_reproduces_linear_fields():
    shape = (8, 4, 6)
    P = CO.level_prolongation(shape, dirichlet_faces=0)
    fine = A_LIN + CO.lattice_nodes(shape).astype(np.float64) @ B_LIN.T
    coarse = A_LIN + (2 * CO.lattice_nodes((4, 2, 3))).astype(np.float64) @ B_LIN.T
    np.testing.assert_allclose(P @ coarse.ravel(), fine.ravel(), rtol=1e-13, atol=1e-13)


def test_l1_jacobi_smoother_spectrum_lies_in_the_unit_interval():
    m, rho, A, f, C = _system(W.config1b())
    H = CO.Hierarchy(m, A)
    for Al, d in zip(H.A, H.d):
        Ad = Al.toarray()
        s = 1.0 / np.sqrt(d)
        lam = np.linalg.eigvalsh(s[:, None] * Ad * s[None, :])
        assert lam.min() > 0 and lam.max() <= 1 + 1e-12


def test_vcycle_is_symmetric_positive_definite():
    m, rho, A, f, C = _system(W.config1b())
    H = CO.Hierarchy(m, A)
    n0 = H.A[0].shape[0]
    rng = np.random.default_rng(11)
    a, b = rng.standard_normal(n0), rng.standard_normal(n0)
    for nu in (1, 2):
        assert a @ H.vcycle(b, nu) == pytest.approx(b @ H.vcycle(a, nu), rel=1e-10)
        assert a @ H.vcycle(a, nu) > 0
    diag = A.diagonal()
    r, s = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    assert r @ H.precondition(diag, s) == pytest.approx(s @ H.precondition(diag, r), rel=1e-10)


def test_coarse_correction_with_an_exact_coarse_solve_is_the_galerkin_projection():
    """On a base grid that is its own coarsest level, P0 V_0(P0^T A u*) = u* for u* = P0 c."""
    dom = W.Domain(4, 2, 2, 2, 0.5)
    w = W.random_field_mesh("tiny_l2", dom, 3, [(0.1, 0.9), (0.4, 0.6)])
    m, rho, A, f, C = _system(w)
    H = CO.Hierarchy(m, A)
    assert H.levels == 1
    c = np.random.default_rng(2).standard_normal(H.P0.shape[1])
    us = H.P0 @ c
    got = H.P0 @ H.vcycle(H.P0.T @ (A @ us))
    assert np.abs(got - us).max() <= 1e-9 * np.abs(us).max()


@pytest.mark.parametrize("name,maker,factor", [("config1b", W.config1b, 3),
                                               ("truss8x4x4L2", lambda: W.small_truss(seed=4, base=(8, 4, 4), L=2), 4)])
def test_twolevel_pcg_reaches_the_direct_solution_in_fewer_iterations(name, maker, factor):
    m, rho, A, f, C = _system(maker())
    u, it2, _ = CO.twolevel_pcg(m, A, f, rtol=1e-8, nu=2)
    it1 = S.jacobi_pcg(A, f, rtol=1e-8)[1]
    assert np.linalg.norm(f - A @ u) <= 1.01e-8 * np.linalg.norm(f)
    ud = S.direct(A, f)
    e = u - ud
    assert np.sqrt(e @ (A @ e) / (ud @ (A @ ud))) <= 1e-6
    assert factor * it2 <= it1


def test_odd_base_grid_coarsens_with_overhanging_cells():
    """A 10x5x5 base (odd y and z counts): the level-1 cells overhang the box; the Galerkin
    operators still equal the quadrature of the coarse basis over the box, the coarse space stays
    in the finite-element space, and the two-level PCG reaches the direct solution in a fraction
    of Jacobi's iterations."""
    dom = W.Domain(10, 5, 5, 1, 0.2)
    w = W.truss_mesh("truss_10x5x5_L1", dom, 3, r0=0.06)
    m, rho, A, f, C = _system(w)
    assert CO.level_shapes(m) == [(10, 5, 5), (5, 3, 3)]
    H = CO.Hierarchy(m, A)
    for level, shape in enumerate(H.shapes):
        K = CO.quadrature_cell_matrices(m, rho, level, w.E0, w.Emin, w.nu, w.penal)
        Aq = CO.assemble_cells(shape, K)
        assert abs(H.A[level] - Aq).max() <= 1e-12 * abs(Aq).max()
    # linear fields: the level prolongation with an overhanging cell stays exact
    P = CO.level_prolongation((10, 5, 5), dirichlet_faces=0)
    fine = A_LIN + CO.lattice_nodes((10, 5, 5)).astype(np.float64) @ B_LIN.T
    coarse = A_LIN + (2 * CO.lattice_nodes((5, 3, 3))).astype(np.float64) @ B_LIN.T
    np.testing.assert_allclose(P @ coarse.ravel(), fine.ravel(), rtol=1e-13, atol=1e-13)
    u, it2, _ = CO.twolevel_pcg(m, A, f, rtol=1e-8, nu=2)
    it1 = S.jacobi_pcg(A, f, rtol=1e-8)[1]
    assert np.linalg.norm(f - A @ u) <= 1.01e-8 * np.linalg.norm(f)
    assert 3 * it2 <= it1
