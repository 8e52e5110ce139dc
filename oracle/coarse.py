"""Oracle of the two-level preconditioner for the reduced system A u = f: a Galerkin coarse
correction on the vertex lattice of the base grid, approximated by a V-cycle over uniform
coarser lattices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's solver is MINRES with Krylov recycling (Sec. 5): the recycled subspace carries
the slowly converging part of the spectrum from one solve to the next.  This module is the
coarse-space counterpart used here instead (an extension with no paper counterpart): the
smooth part of the error is removed by a projection onto a fixed coarse space.  Every choice
below is a reading made for it:

* **Levels.**  Level 0 is the vertex lattice of the base grid: ``(nx+1)(ny+1)(nz+1)`` nodes at
  the base-cell corners, cell side ``h0``.  Level l+1 has ``ceil(n / 2)`` cells per axis for the
  ``n`` of level l, cells of twice the side anchored at the origin; a level is added while the
  current one has more than 64 cells.  With an odd count the last coarse cell overhangs the box;
  the coarse functions restricted to the box stay trilinear on every finer cell, so the levels
  stay nested.  An axis whose upper face is clamped is halved only while its count is even (the
  clamped face must stay a lattice plane); an odd count there ends the hierarchy.  The last
  level is the coarsest.
* **Unknowns.**  Three displacement components per lattice node (DOF ``3 I + c``, nodes
  numbered with x fastest); nodes on a clamped face (the mesh's Dirichlet faces) carry none.
* **Fine -> level 0 (P0).**  The trilinear interpolant of the lattice values, evaluated at the
  free nodes of the mesh.  Every leaf lies inside one base cell, so each coarse function is
  trilinear on each leaf and agrees with the hanging-node interpolation (Eq. 6): the coarse
  space is a subspace of the finite-element space.
* **Level l -> l+1 (P).**  Nodal interpolation between nested uniform lattices (weights 1,
  1/2, 1/4, 1/8).
* **Operators.**  Galerkin: ``A0 = P0^T A P0`` and ``A_{l+1} = P^T A_l P``.
* **Smoother.**  l1-Jacobi, ``x += d^-1 (b - A_l x)`` with ``d_i = sum_j |A_l[i, j]|``; it needs
  no eigenvalue estimate and converges for every SPD matrix.
* **Cycle.**  ``V_l(b)``: ``nu`` sweeps from zero, the residual restricted by ``P^T``,
  ``V_{l+1}`` of it prolongated by ``P`` and added, then ``nu`` sweeps; on the coarsest level
  a direct solve.  Pre- and post-smoothing are the same symmetric sweeps, so ``V_0`` is a
  fixed symmetric positive definite operator.
* **Preconditioner.**  Additive: ``M^-1 r = D^-1 r + P0 V_0(P0^T r)`` with D the diagonal of A
  (the Jacobi preconditioner of Sec. 5 plus the coarse correction).

The plain definitions are written out (sparse products, explicit sweeps); the tests pin them
against an independent quadrature of the coarse basis, exactness on linear fields and the
algebraic properties of the cycle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem as F
from .mesh import Mesh


# ---------------------------------------------------------------- lattices
def level_shapes(mesh: Mesh, dirichlet_faces: int = 1):
    """Cell counts (X, Y, Z) of the levels 0, 1, ... (rule in the module docstring)."""
    shapes = [(mesh.nx, mesh.ny, mesh.nz)]
    while True:
        cur = shapes[-1]
        if cur[0] * cur[1] * cur[2] <= 64:
            return shapes
        if any(cur[a] % 2 and (dirichlet_faces >> (2 * a + 1)) & 1 for a in range(3)):
            return shapes
        shapes.append(tuple((n + 1) // 2 for n in cur))


def lattice_nodes(shape):
    """(n, 3) lattice coordinates of the nodes of a level with `shape` cells, x fastest."""
    X, Y, Z = shape
    k, j, i = np.meshgrid(np.arange(Z + 1), np.arange(Y + 1), np.arange(X + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], 1)


def lattice_free(shape, dirichlet_faces: int) -> np.ndarray:
    """Free lattice nodes (not on a clamped face), ascending."""
    p = lattice_nodes(shape)
    ext = np.array(shape)
    fixed = np.zeros(len(p), bool)
    for f in range(6):
        if (dirichlet_faces >> f) & 1:
            a, side = f // 2, f % 2
            fixed |= p[:, a] == (ext[a] if side else 0)
    return np.nonzero(~fixed)[0]


def _dofs(nodes):
    return (3 * np.asarray(nodes)[:, None] + np.arange(3)).ravel()


# ---------------------------------------------------------------- transfers
def fine_prolongation(mesh: Mesh, dirichlet_faces: int = 1) -> sp.csr_matrix:
    """P0 (free fine DOFs x free level-0 DOFs): trilinear interpolation of the base-lattice
    values at the free mesh nodes, per component."""
    S = 1 << mesh.L
    X, Y, Z = mesh.nx, mesh.ny, mesh.nz
    fn = F.free_nodes(mesh)
    p = mesh.nodes[fn].astype(np.int64)
    cell = np.minimum(p // S, np.array([X - 1, Y - 1, Z - 1]))
    t = (p - cell * S) / S                          # local coordinates in [0, 1]
    rows, cols, vals = [], [], []
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = ((t[:, 0] if a else 1 - t[:, 0]) * (t[:, 1] if b else 1 - t[:, 1])
                     * (t[:, 2] if c else 1 - t[:, 2]))
                J = (cell[:, 0] + a) + (X + 1) * ((cell[:, 1] + b) + (Y + 1) * (cell[:, 2] + c))
                keep = w != 0
                rows.append(np.nonzero(keep)[0])
                cols.append(J[keep])
                vals.append(w[keep])
    Pn = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(fn.size, (X + 1) * (Y + 1) * (Z + 1)))
    Pn = Pn[:, lattice_free((X, Y, Z), dirichlet_faces)]
    return sp.kron(Pn, sp.eye(3)).tocsr()


def level_prolongation(shape, dirichlet_faces: int = 1) -> sp.csr_matrix:
    """P (free DOFs of the level with `shape` cells x free DOFs of the next, halved level):
    nodal interpolation between nested lattices."""
    X, Y, Z = shape
    Xc, Yc, Zc = (X + 1) // 2, (Y + 1) // 2, (Z + 1) // 2
    p = lattice_nodes(shape)

    def axis(i):
        lo = i // 2
        odd = i % 2 == 1
        return [(lo, np.where(odd, 0.5, 1.0)), (lo + 1, np.where(odd, 0.5, 0.0))]

    rows, cols, vals = [], [], []
    idx = np.arange(len(p))
    for ia, wa in axis(p[:, 0]):
        for ib, wb in axis(p[:, 1]):
            for ic, wc in axis(p[:, 2]):
                w = wa * wb * wc
                keep = w != 0
                rows.append(idx[keep])
                cols.append((ia + (Xc + 1) * (ib + (Yc + 1) * ic))[keep])
                vals.append(w[keep])
    T = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(len(p), (Xc + 1) * (Yc + 1) * (Zc + 1)))
    T = T[lattice_free(shape, dirichlet_faces)][:, lattice_free((Xc, Yc, Zc), dirichlet_faces)]
    return sp.kron(T, sp.eye(3)).tocsr()


# ---------------------------------------------------------------- the hierarchy and the cycle
def l1_diagonal(A: sp.spmatrix) -> np.ndarray:
    """d_i = sum_j |A[i, j]| (the l1-Jacobi smoother's diagonal)."""
    return np.asarray(abs(A).sum(axis=1)).ravel()


class Hierarchy:
    """Galerkin operators of all levels for the reduced matrix A of `mesh`."""

    def __init__(self, mesh: Mesh, A: sp.spmatrix, dirichlet_faces: int = 1):
        self.shapes = level_shapes(mesh, dirichlet_faces)
        self.P0 = fine_prolongation(mesh, dirichlet_faces)
        self.A = [(self.P0.T @ A @ self.P0).tocsr()]
        self.P = []
        for s in self.shapes[:-1]:
            Pl = level_prolongation(s, dirichlet_faces)
            self.P.append(Pl)
            self.A.append((Pl.T @ self.A[-1] @ Pl).tocsr())
        self.d = [l1_diagonal(Al) for Al in self.A]
        self.lu = spla.splu(self.A[-1].tocsc())

    @property
    def levels(self):
        return len(self.A)

    def vcycle(self, b, nu: int = 2, level: int = 0):
        """V_level(b) (module docstring); on the coarsest level a direct solve."""
        b = np.asarray(b, np.float64)
        if level == self.levels - 1:
            return self.lu.solve(b)
        A, d = self.A[level], self.d[level]
        x = b / d
        for _ in range(nu - 1):
            x = x + (b - A @ x) / d
        r = b - A @ x
        Pl = self.P[level]
        x = x + Pl @ self.vcycle(Pl.T @ r, nu, level + 1)
        for _ in range(nu):
            x = x + (b - A @ x) / d
        return x

    def precondition(self, A_diag, r, nu: int = 2):
        """M^-1 r = D^-1 r + P0 V_0(P0^T r)."""
        r = np.asarray(r, np.float64)
        return r / A_diag + self.P0 @ self.vcycle(self.P0.T @ r, nu)


def twolevel_pcg(mesh: Mesh, A: sp.spmatrix, f, u0=None, rtol=1e-8, nu: int = 2, dirichlet_faces: int = 1,
                 max_iter=100000):
    """PCG with the additive two-level preconditioner.  Returns (u, iterations, residual)."""
    from . import solve as S
    H = Hierarchy(mesh, A, dirichlet_faces)
    diag = A.diagonal()
    return S.pcg(A, f, lambda r: H.precondition(diag, r, nu), u0, rtol, max_iter)


# ---------------------------------------------------------------- independent check
def quadrature_cell_matrices(mesh: Mesh, rho, level: int = 0, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0,
                             dirichlet_faces: int = 1):
    """(cells, 24, 24): the stiffness of the level's trilinear cell basis with the mesh's
    piecewise-constant Young's modulus, K_C = sum over leaves e in C of E_e * integral over e of
    B_C^T D B_C, each integral by 2x2x2 Gauss points of the leaf (exact: the integrand has
    degree <= 2 per axis).  A direct quadrature of the coarse basis, independent of K0, of the
    constraint map and of any prolongation; local DOF 3 k + c of cell corner k = i + 2j + 4m."""
    X, Y, Z = level_shapes(mesh, dirichlet_faces)[level]
    S = (1 << mesh.L) << level                  # cell side in finest units
    H = mesh.h0 * (1 << level)
    D = F.elasticity_matrix(1.0, nu)
    E = F.young(rho, E0, Emin, penal)
    g = 1.0 / np.sqrt(3.0)
    gp = np.array([(1 - g) / 2, (1 + g) / 2])
    K = np.zeros((X * Y * Z, 24, 24))
    for e in range(mesh.Ne):
        ix, iy, iz, lv = (int(v) for v in mesh.leaves[e])
        s = 1 << (mesh.L - lv)
        cell = np.array([ix // S, iy // S, iz // S])
        ci = cell[0] + X * (cell[1] + Y * cell[2])
        lo = (np.array([ix, iy, iz]) - cell * S) / S
        side = s / S
        wvol = (side ** 3) / 8.0                 # Gauss weight of the leaf in cell coordinates
        for a in gp:
            for b in gp:
                for c in gp:
                    xi = lo + side * np.array([a, b, c])
                    B = F.strain_matrix(xi) / H  # gradients of the cell basis in physical units
                    K[ci] += E[e] * (B.T @ D @ B) * wvol * H ** 3
    return K


def assemble_cells(shape, K, dirichlet_faces: int = 1) -> sp.csr_matrix:
    """The free-DOF matrix sum_C K_C of a level from its cell matrices."""
    X, Y, Z = shape
    rows, cols, vals = [], [], []
    for ci in range(X * Y * Z):
        i, j, k = ci % X, (ci // X) % Y, ci // (X * Y)
        corners = [(i + (q & 1)) + (X + 1) * ((j + ((q >> 1) & 1)) + (Y + 1) * (k + (q >> 2))) for q in range(8)]
        dof = _dofs(corners)
        rows.append(np.repeat(dof, 24))
        cols.append(np.tile(dof, 24))
        vals.append(K[ci].ravel())
    n = 3 * (X + 1) * (Y + 1) * (Z + 1)
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    free = _dofs(lattice_free(shape, dirichlet_faces))
    return M[free][:, free].tocsr()
