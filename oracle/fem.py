"""Oracle finite-element operators: K0, K(rho), the constraint map C and the
reduced system (paper Sec. 3 Eq. 1-2, Sec. 6 Eq. 6-9).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* B8 element: trilinear displacement, constant density per element (Sec. 3).
* K0 is the stiffness of the unit cube for E = 1 and Poisson ratio nu with the
  isotropic elasticity matrix, integrated by 2x2x2 Gauss quadrature (exact for
  the affine cube).  Local DOF ``3 k + c`` is component c of corner k.
* An element of side h has stiffness ``h * K0`` (B scales as 1/h, the volume as
  h^3) and Young's modulus ``E_e = Emin + rho_e^p (E0 - Emin)``; Emin = 0 is the
  paper's Eq. 2 exactly.
* Hanging DOFs are eliminated through ``u_full = C u`` where C is the identity
  on free DOFs, the interpolation P on hanging DOFs (Eq. 6) and zero on
  Dirichlet DOFs; the reduced matrix is ``A = C^T K C`` and the load is
  ``f = C^T f_full``.  The paper's Eq. 8 keeps the constrained rows with a unit
  diagonal instead; its solution restricted to free DOFs is the same vector and
  Eq. 9 recovers the same ``u_full`` (this equivalence is a test).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import CORNER_OFFSETS, Mesh


def elasticity_matrix(E: float, nu: float) -> np.ndarray:
    """Isotropic D in Voigt order (xx, yy, zz, xy, yz, zx), engineering shear strains."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_gradients(xi: np.ndarray) -> np.ndarray:
    """d N_k / d(x, y, z) of the 8 trilinear shape functions on [0,1]^3 at point xi: (8, 3)."""
    g = np.zeros((8, 3))
    for k, (i, j, m) in enumerate(CORNER_OFFSETS):
        f = [xi[0] if i else 1 - xi[0], xi[1] if j else 1 - xi[1], xi[2] if m else 1 - xi[2]]
        d = [1.0 if i else -1.0, 1.0 if j else -1.0, 1.0 if m else -1.0]
        g[k, 0] = d[0] * f[1] * f[2]
        g[k, 1] = f[0] * d[1] * f[2]
        g[k, 2] = f[0] * f[1] * d[2]
    return g


def strain_matrix(xi: np.ndarray) -> np.ndarray:
    """B (6 x 24) with strain = B u_e."""
    g = shape_gradients(xi)
    B = np.zeros((6, 24))
    for k in range(8):
        gx, gy, gz = g[k]
        c = 3 * k
        B[0, c + 0] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 0] = gy
        B[3, c + 1] = gx
        B[4, c + 1] = gz
        B[4, c + 2] = gy
        B[5, c + 0] = gz
        B[5, c + 2] = gx
    return B


def reference_stiffness(nu: float) -> np.ndarray:
    """K0 = sum over the 2x2x2 Gauss points of B^T D B * weight, unit cube, E = 1."""
    D = elasticity_matrix(1.0, nu)
    g = 1.0 / np.sqrt(3.0)
    pts = [(1 - g) / 2, (1 + g) / 2]
    K0 = np.zeros((24, 24))
    for a in pts:
        for b in pts:
            for c in pts:
                B = strain_matrix(np.array([a, b, c]))
                K0 += B.T @ D @ B * 0.125
    return K0


def young(rho, E0, Emin, penal):
    return Emin + np.asarray(rho) ** penal * (E0 - Emin)


def element_dofs(mesh: Mesh) -> np.ndarray:
    """(Ne, 24) global full-space DOF indices 3*node + component."""
    return (3 * mesh.conn[:, :, None] + np.arange(3)[None, None, :]).reshape(mesh.Ne, 24)


def assemble_full(mesh: Mesh, rho, E0, Emin, nu, penal) -> sp.csr_matrix:
    """K_full = sum_e E_e h_e K0 scattered by the element DOFs (no constraints)."""
    K0 = reference_stiffness(nu)
    ce = young(rho, E0, Emin, penal) * mesh.h
    dofs = element_dofs(mesh)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    vals = (ce[:, None, None] * K0[None]).ravel()
    n = 3 * mesh.Nn
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def free_nodes(mesh: Mesh) -> np.ndarray:
    """Nodes that carry unknowns: neither hanging nor Dirichlet, ascending."""
    hang = np.zeros(mesh.Nn, bool)
    hang[mesh.hanging_ids()] = True
    return np.nonzero(~hang & ~mesh.dirichlet)[0]


def constraint_matrix(mesh: Mesh) -> sp.csr_matrix:
    """C (3 Nn x n): free DOFs identity, hanging DOFs interpolate their masters (Eq. 6),
    Dirichlet DOFs zero (homogeneous prescribed displacement)."""
    fn = free_nodes(mesh)
    col_of = -np.ones(mesh.Nn, np.int64)
    col_of[fn] = np.arange(fn.size)
    rows, cols, vals = [], [], []
    for c in range(3):
        rows.append(3 * fn + c)
        cols.append(3 * np.arange(fn.size) + c)
        vals.append(np.ones(fn.size))
    for h, masters in mesh.hanging.items():
        if mesh.dirichlet[h]:
            continue
        for m, w in masters:
            if col_of[m] < 0:
                continue          # a Dirichlet master contributes its prescribed zero
            for c in range(3):
                rows.append(np.array([3 * h + c]))
                cols.append(np.array([3 * col_of[m] + c]))
                vals.append(np.array([float(w)]))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.coo_matrix((vals, (rows, cols)), shape=(3 * mesh.Nn, 3 * fn.size)).tocsr()


def full_load(mesh: Mesh, load_nodes, load_comp, load_val) -> np.ndarray:
    """Nodal force vector on all 3 Nn DOFs; each load must sit on a mesh node."""
    f = np.zeros(3 * mesh.Nn)
    lookup = {tuple(p): i for i, p in enumerate(map(tuple, mesh.nodes))}
    for p, c, v in zip(np.asarray(load_nodes), np.asarray(load_comp), np.asarray(load_val)):
        key = tuple(int(t) for t in p)
        if key not in lookup:
            raise ValueError(f"load point {key} is not a mesh node")
        f[3 * lookup[key] + int(c)] += v
    return f


def reduced_system(mesh: Mesh, rho, load_nodes, load_comp, load_val, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0):
    """(A, f, C) with A = C^T K(rho) C and f = C^T f_full (Eq. 7 with constrained DOFs eliminated)."""
    K = assemble_full(mesh, rho, E0, Emin, nu, penal)
    C = constraint_matrix(mesh)
    A = (C.T @ K @ C).tocsr()
    A.sum_duplicates()
    f = C.T @ full_load(mesh, load_nodes, load_comp, load_val)
    return A, f, C


def to_full_layout(mesh: Mesh, v_free: np.ndarray) -> np.ndarray:
    """Embed a free-DOF vector into the 3 Nn layout with zeros on constrained DOFs."""
    out = np.zeros(3 * mesh.Nn)
    fn = free_nodes(mesh)
    out.reshape(-1, 3)[fn] = np.asarray(v_free).reshape(-1, 3)
    return out


def from_full_layout(mesh: Mesh, v_full: np.ndarray) -> np.ndarray:
    return np.asarray(v_full).reshape(-1, 3)[free_nodes(mesh)].ravel()


def operator_rows(mesh: Mesh, rho, x_full, nodes, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0, absolute=False):
    """(C^T K(rho) C x) at the given (free) nodes, element by element, for meshes too large to
    assemble: x_full is an A-space vector (3 Nn, constrained entries ignored).  With `absolute`
    every factor is replaced by its absolute value, giving the rounding scale (|A| |x|)."""
    K0 = reference_stiffness(nu)
    if absolute:
        K0 = np.abs(K0)
    x = np.asarray(x_full, np.float64).reshape(-1, 3)
    if absolute:
        x = np.abs(x)
    ce = young(rho, E0, Emin, penal) * mesh.h
    hang = mesh.hanging
    # node -> (element, corner) incidences, and master -> hanging nodes
    order = np.argsort(mesh.conn.ravel(), kind="stable")
    flat = mesh.conn.ravel()[order]
    starts = np.searchsorted(flat, np.arange(mesh.Nn + 1))
    of_master = {}
    for h, ms in hang.items():
        for mm, w in ms:
            of_master.setdefault(mm, []).append((h, float(w)))

    def corner_value(n):
        if mesh.dirichlet[n]:
            return np.zeros(3)
        if n in hang:
            v = np.zeros(3)
            for mm, w in hang[n]:
                if not mesh.dirichlet[mm]:
                    v += float(w) * x[mm]
            return v
        return x[n]

    def element_result(e):
        X = np.concatenate([corner_value(n) for n in mesh.conn[e]])
        return (ce[e] * (K0 @ X)).reshape(8, 3)

    out = np.zeros((len(nodes), 3))
    for i, t in enumerate(nodes):
        t = int(t)
        acc = np.zeros(3)
        terms = [(t, 1.0)] + of_master.get(t, [])
        for n, w in terms:
            for pos in order[starts[n]:starts[n + 1]]:
                e, k = divmod(int(pos), 8)
                acc += w * element_result(e)[k]
        out[i] = acc
    return out
