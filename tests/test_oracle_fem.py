"""Pins for the oracle's element matrix, assembly and constraint elimination
(paper Sec. 3 Eq. 1-2, Sec. 6 Eq. 6-9)."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fem as F
from oracle import mesh as M
from oracle import solve as S

NU = 0.3


def _exact_k0(nu: Fraction):
    """K0 by exact separable integration of polynomials on [0,1]^3 (no quadrature).

    For corner k = (i, j, m): N_k = f_i(x) f_j(y) f_m(z) with f_0 = 1 - t, f_1 = t.
    1D integrals: int f_a f_b = 1/3 (a == b) or 1/6; int f_a' f_b = s_a / 2; int f_a' f_b' = s_a s_b,
    with s_0 = -1, s_1 = +1."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = Fraction(1, 2) / (1 + nu)
    Dm = [[Fraction(0)] * 6 for _ in range(6)]
    for a in range(3):
        for b in range(3):
            Dm[a][b] = lam + (2 * mu if a == b else 0)
    for a in range(3, 6):
        Dm[a][a] = mu
    # strain p, displacement component c -> derivative axis (Voigt, engineering shear)
    deriv = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (3, 0): 1, (3, 1): 0, (4, 1): 2, (4, 2): 1, (5, 0): 2, (5, 2): 0}
    s = [-1, 1]

    def i1(a, b, da, db):
        if da and db:
            return Fraction(s[a] * s[b])
        if da:
            return Fraction(s[a], 2)
        if db:
            return Fraction(s[b], 2)
        return Fraction(1, 3) if a == b else Fraction(1, 6)

    corners = [(k & 1, (k >> 1) & 1, (k >> 2) & 1) for k in range(8)]
    K = [[Fraction(0)] * 24 for _ in range(24)]
    for ka, A in enumerate(corners):
        for ca in range(3):
            for kb, B in enumerate(corners):
                for cb in range(3):
                    tot = Fraction(0)
                    for p in range(6):
                        if (p, ca) not in deriv:
                            continue
                        for q in range(6):
                            if (q, cb) not in deriv or Dm[p][q] == 0:
                                continue
                            ax_a, ax_b = deriv[(p, ca)], deriv[(q, cb)]
                            v = Fraction(1)
                            for ax in range(3):
                                v *= i1(A[ax], B[ax], ax == ax_a, ax == ax_b)
                            tot += Dm[p][q] * v
                    K[3 * ka + ca][3 * kb + cb] = tot
    return K


def _rigid_modes():
    X = M.CORNER_OFFSETS.astype(np.float64)
    modes = []
    for c in range(3):
        v = np.zeros((8, 3))
        v[:, c] = 1
        modes.append(v.ravel())
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1
        modes.append(np.cross(w, X).ravel())
    return np.array(modes).T


def test_k0_matches_exact_rational_integration():
    K0 = F.reference_stiffness(NU)
    Kx = _exact_k0(Fraction(3, 10))
    Kx = np.array([[float(v) for v in row] for row in Kx])
    assert np.abs(K0 - Kx).max() <= 4e-16 * np.abs(Kx).max() * 24


def test_k0_symmetric_with_six_rigid_body_null_modes():
    K0 = F.reference_stiffness(NU)
    assert np.abs(K0 - K0.T).max() < 1e-16
    ev = np.linalg.eigvalsh(K0)
    assert np.all(np.abs(ev[:6]) < 1e-14)
    assert np.all(ev[6:] > 1e-2)
    R = _rigid_modes()
    assert np.abs(K0 @ R).max() < 1e-14


def test_k0_uniform_strain_energy_closed_form():
    K0 = F.reference_stiffness(NU)
    D = F.elasticity_matrix(1.0, NU)
    X = M.CORNER_OFFSETS.astype(np.float64)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((3, 3))
    u = (X @ G.T).ravel()                     # u = G x, strain = sym(G)
    eps = np.array([G[0, 0], G[1, 1], G[2, 2], G[0, 1] + G[1, 0], G[1, 2] + G[2, 1], G[2, 0] + G[0, 2]])
    assert np.isclose(0.5 * u @ K0 @ u, 0.5 * eps @ D @ eps, rtol=1e-13)


def test_element_stiffness_scales_linearly_with_size():
    # A cube of side h under u = G x stores energy h^3 * (1/2) eps.D.eps; with nodal values
    # scaled by h the quadratic form h * u^T K0 u must reproduce that.
    K0 = F.reference_stiffness(NU)
    D = F.elasticity_matrix(1.0, NU)
    G = np.array([[0.2, 0.1, 0.0], [0.0, -0.1, 0.3], [0.05, 0.0, 0.1]])
    eps = np.array([G[0, 0], G[1, 1], G[2, 2], G[0, 1] + G[1, 0], G[1, 2] + G[2, 1], G[2, 0] + G[0, 2]])
    for h in (0.25, 1 / 24, 3.0):
        u = ((h * M.CORNER_OFFSETS) @ G.T).ravel()
        assert np.isclose(0.5 * h * u @ K0 @ u, h ** 3 * 0.5 * eps @ D @ eps, rtol=1e-13)


def _mesh(w, faces=None):
    d = w.dom
    faces = w.dirichlet_faces if faces is None else faces
    return M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=faces)


def test_patch_test_general_linear_field_without_supports():
    """No Dirichlet faces: any linear u = G x + b is stress-uniform, so C^T K C u vanishes at every
    node off the box surface, hanging masters included."""
    w = W.config1b()
    m = _mesh(w, faces=0)
    K = F.assemble_full(m, np.ones(m.Ne), 1.0, 0.0, NU, 3.0)
    C = F.constraint_matrix(m)
    fn = F.free_nodes(m)
    assert fn.size == m.Nn - len(m.hanging)
    G = np.array([[0.1, 0.02, -0.03], [0.01, -0.2, 0.05], [0.04, 0.0, 0.15]])
    X = m.nodes * (w.dom.h0 / (1 << w.dom.L))
    u = X @ G.T + np.array([0.3, -0.1, 0.2])
    uf = C @ u[fn].ravel()
    assert np.abs(uf - u.ravel()).max() < 1e-14
    r = (C.T @ (K @ uf)).reshape(-1, 3)
    ext = np.array([w.dom.nx, w.dom.ny, w.dom.nz]) << w.dom.L
    interior = ((m.nodes[fn] > 0) & (m.nodes[fn] < ext)).all(axis=1)
    assert interior.sum() > 10
    assert np.abs(r[interior]).max() < 1e-13
    # and the rigid part alone produces no force anywhere
    W_ = np.array([[0.0, 0.3, -0.2], [-0.3, 0.0, 0.1], [0.2, -0.1, 0.0]])
    ur = (X @ W_.T + 0.5).ravel()
    assert np.abs(C.T @ (K @ (C @ ur.reshape(-1, 3)[fn].ravel()))).max() < 1e-13


def test_patch_test_uniform_strain_across_hanging_nodes():
    w = W.config1b()
    m = _mesh(w)
    rho = np.ones(m.Ne)
    K = F.assemble_full(m, rho, 1.0, 0.0, NU, 3.0)
    C = F.constraint_matrix(m)
    fn = F.free_nodes(m)
    # a uniform strain that vanishes on the clamped face x = 0: u = x g
    g = np.array([0.1, 0.02, -0.03])
    X = m.nodes * (w.dom.h0 / (1 << w.dom.L))
    u = X[:, :1] * g[None, :]
    ut = u[fn].ravel()
    uf = C @ ut
    # hanging DOFs reproduce the linear field
    assert np.abs(uf.reshape(-1, 3) - u).max() < 1e-15
    # internal equilibrium: at free nodes off the box surface the reduced residual vanishes
    ext = np.array([w.dom.nx, w.dom.ny, w.dom.nz]) << w.dom.L
    r = (C.T @ (K @ u.ravel())).reshape(-1, 3)
    interior = ((m.nodes[fn] > 0) & (m.nodes[fn] < ext)).all(axis=1)
    assert interior.sum() > 10
    scale = np.abs(K @ u.ravel()).max()
    assert np.abs(r[interior]).max() < 1e-12 * max(scale, 1.0)


def test_reduced_matrix_equals_dense_bruteforce():
    w = W.config1()
    m = _mesh(w)
    rho = w.rho[m.perm]
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val)
    # dense: element loop, then explicit elimination through a dense C built from the table
    K0 = F.reference_stiffness(NU)
    n = 3 * m.Nn
    K = np.zeros((n, n))
    E = F.young(rho, 1.0, 1e-9, 3.0)
    for e in range(m.Ne):
        dofs = (3 * m.conn[e][:, None] + np.arange(3)).ravel()
        K[np.ix_(dofs, dofs)] += E[e] * m.h[e] * K0
    fn = F.free_nodes(m)
    col = {int(v): i for i, v in enumerate(fn)}
    Cd = np.zeros((n, 3 * fn.size))
    for i in fn:
        for c in range(3):
            Cd[3 * i + c, 3 * col[int(i)] + c] = 1
    for h, ms in m.hanging.items():
        if m.dirichlet[h]:
            continue
        for j, wt in ms:
            if int(j) in col:
                for c in range(3):
                    Cd[3 * h + c, 3 * col[int(j)] + c] += float(wt)
    Ad = Cd.T @ K @ Cd
    assert np.abs(A.toarray() - Ad).max() <= 1e-13 * np.abs(Ad).max()
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(Ad).max()


def test_eq8_unit_diagonal_form_gives_the_same_displacement():
    """Eq. 8 keeps constrained DOFs with unit diagonal; Eq. 9 recovers u. Same u as elimination."""
    w = W.config1()
    m = _mesh(w)
    rho = w.rho[m.perm]
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val)
    u = S.direct(A, f)
    uf = C @ u
    # paper's form on all 3 Nn DOFs: group one = free, group two = hanging + Dirichlet
    K = F.assemble_full(m, rho, 1.0, 1e-9, NU, 3.0)
    fn = F.free_nodes(m)
    n = 3 * m.Nn
    import scipy.sparse as sp
    fdofs = (3 * fn[:, None] + np.arange(3)).ravel()
    Sel = sp.csr_matrix((np.ones(fdofs.size), (np.arange(fdofs.size), fdofs)), shape=(fdofs.size, n))
    Qfull = (C @ Sel).tocsr()          # [I 0; P 0] on the full space
    fullf = F.full_load(m, w.load_nodes, w.load_comp, w.load_val)
    constrained = np.ones(n, bool)
    constrained[fdofs] = False
    Afull = (Qfull.T @ K @ Qfull + sp.diags(constrained.astype(float))).tocsc()
    uhat = spla.splu(Afull).solve(Qfull.T @ fullf)
    assert np.abs(uhat[constrained]).max() == 0.0
    u9 = Qfull @ uhat
    assert np.abs(u9 - uf).max() <= 1e-9 * np.abs(uf).max()


def test_operator_rows_match_assembled_operator():
    """The element-by-element row evaluation used for meshes too large to assemble."""
    w = W.config1b()
    m = _mesh(w)
    rho = w.rho[m.perm]
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val)
    x = np.random.default_rng(0).standard_normal(3 * m.Nn)
    fn = F.free_nodes(m)
    y = (A @ F.from_full_layout(m, x)).reshape(-1, 3)
    rows = F.operator_rows(m, rho, x, fn[::5])
    assert np.abs(rows - y[::5]).max() <= 1e-14 * np.abs(y).max()
    absrows = F.operator_rows(m, rho, x, fn[::5], absolute=True)
    yabs = (abs(A) @ np.abs(F.from_full_layout(m, x))).reshape(-1, 3)
    assert np.all(absrows >= np.abs(rows) - 1e-15)
    assert np.all(absrows >= yabs[::5] * (1 - 1e-13))   # |C^T||K||C||x| bounds |A||x|
