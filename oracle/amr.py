"""Oracle of the dynamic mesh adaptation (paper Sec. 4) and the design difference (Eq. 10).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings (the paper states the rules in words only):

* Marking (Sec. 4, step 1): element e is *solid* when rho_e >= rho_s.  It is marked
  for refinement (+1) when it is solid or some solid element lies at a distance
  below r_AMR (distance between element centres, as for the filter); otherwise it
  is void with no solid element that close and is marked for derefinement (-1).  An
  element at the finest level cannot be refined (0), one at level 0 cannot be
  derefined (0).  The distance test is exact: centres in half finest-cell units are
  integers, and dist < r is taken as d2 < (2 r / unit)^2 with d2 their integer
  squared distance (centres exactly r apart are common, e.g. r = 2 finest cells).
* Sweep 1: a -1 mark survives only if all 8 siblings (the children of the same
  parent) are leaves marked -1.
* Sweep 2: a -1 mark survives only if the coarsened parent (level l-1) would differ
  by at most one level from every leaf whose closure meets the parent box, taking
  each such leaf at its level after its own refinement (level + 1 when marked +1)
  and ignoring other coarsenings (a conservative, order-independent reading of
  "would lead to level two or higher incompatibility").
* New mesh: +1 leaves split into 8, surviving -1 families merge into their parent,
  then leaves are refined until the mesh is 2:1 balanced ("refine the gray
  elements", Sec. 6).  Children inherit the parent density; a merged parent takes
  the mean of its 8 children (summed in sibling order, x fastest), so that the
  integral of rho over the box is unchanged.
* Eq. 10: D(rho1, rho2) = int |rho1 - rho2| / int rho1, both designs sampled on
  the finest grid (every cell takes the density of the leaf covering it).
* Displacement transfer to an adapted mesh (the warm start after remeshing; the paper
  maps the solution onto the updated mesh): the old finite-element field -- trilinear
  on each old leaf, hanging values interpolated -- evaluated at the new nodes.  The
  field is continuous, so any old leaf whose closed box contains a point gives its
  value; the leaf covering the finest cell at the point's coordinates, clamped to the
  box, is used.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .mesh import Mesh, leaf_owner_map


def _half_cell_centres(mesh: Mesh) -> np.ndarray:
    """Element centres in units of half a finest cell: exact integers 2 * anchor + size."""
    return 2 * mesh.leaves[:, :3].astype(np.int64) + mesh.size[:, None]


def _threshold(mesh: Mesh, r_amr: float) -> float:
    """(2 r / unit)^2: 'distance below r' is 'squared half-cell distance below this'."""
    t = 2.0 * r_amr / (mesh.h0 / (1 << mesh.L))
    return t * t


def _finish(mesh: Mesh, refine) -> np.ndarray:
    m = np.where(refine, 1, -1).astype(np.int8)
    lvl = mesh.leaves[:, 3]
    m[(m == 1) & (lvl >= mesh.L)] = 0
    m[(m == -1) & (lvl == 0)] = 0
    return m


def mark(mesh: Mesh, rho, rho_solid: float, r_amr: float) -> np.ndarray:
    rho = np.asarray(rho, np.float64)
    solid = rho >= rho_solid
    c2 = _half_cell_centres(mesh)
    near = np.zeros(mesh.Ne, bool)
    if solid.any():
        # nearest solid centre (exact: integer coordinates), then the exact squared distance
        tree = cKDTree(c2[solid].astype(np.float64))
        _, j = tree.query(c2.astype(np.float64), k=1)
        diff = c2 - c2[solid][j]
        near = (diff * diff).sum(axis=1).astype(np.float64) < _threshold(mesh, r_amr)
    return _finish(mesh, solid | near)


def mark_bruteforce(mesh: Mesh, rho, rho_solid: float, r_amr: float) -> np.ndarray:
    c2 = _half_cell_centres(mesh)
    thr = _threshold(mesh, r_amr)
    refine = np.zeros(mesh.Ne, bool)
    for e in range(mesh.Ne):
        refine[e] = rho[e] >= rho_solid
        for d in range(mesh.Ne):
            if rho[d] >= rho_solid:
                dd = [int(c2[e, a] - c2[d, a]) for a in range(3)]
                if float(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]) < thr:
                    refine[e] = True
    return _finish(mesh, refine)


def _parent(leaf, L):
    s = 1 << (L - int(leaf[3]))
    return tuple(int(v) // (2 * s) * (2 * s) for v in leaf[:3]), 2 * s


def leaf_index(mesh: Mesh) -> dict:
    """(anchor, level) -> element index."""
    return {(tuple(int(v) for v in lf[:3]), int(lf[3])): i for i, lf in enumerate(mesh.leaves)}


def family_marked(mesh: Mesh, index: dict, marks, e: int) -> bool:
    """Sweep 1 predicate: all 8 children of e's parent are leaves marked -1."""
    lf = mesh.leaves[e]
    pa, ps = _parent(lf, mesh.L)
    s = ps // 2
    for k in range(8):
        a = (pa[0] + s * (k & 1), pa[1] + s * ((k >> 1) & 1), pa[2] + s * ((k >> 2) & 1))
        j = index.get((a, int(lf[3])))
        if j is None or marks[j] != -1:
            return False
    return True


def parent_compatible(mesh: Mesh, owner, marks, e: int) -> bool:
    """Sweep 2 predicate: every leaf whose closure meets the parent box of e ends (after its own
    refinement) at most one level finer than that parent (level l - 1), i.e. at level <= l."""
    lf = mesh.leaves[e]
    pa, ps = _parent(lf, mesh.L)
    lo = np.maximum(np.array(pa) - 1, 0)
    hi = np.minimum(np.array(pa) + ps + 1, np.array(owner.shape))
    touching = np.unique(owner[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
    new_level = mesh.leaves[touching, 3] + (np.asarray(marks)[touching] == 1)
    return bool(new_level.max() <= int(lf[3]))


def sweep_siblings(mesh: Mesh, marks) -> np.ndarray:
    index = leaf_index(mesh)
    out = np.array(marks, np.int8)
    for e in np.nonzero(np.asarray(marks) == -1)[0]:
        if not family_marked(mesh, index, marks, int(e)):
            out[e] = 0
    return out


def sweep_balance(mesh: Mesh, marks) -> np.ndarray:
    owner = leaf_owner_map(mesh.nx, mesh.ny, mesh.nz, mesh.L, mesh.leaves)
    out = np.array(marks, np.int8)
    for e in np.nonzero(np.asarray(marks) == -1)[0]:
        if not parent_compatible(mesh, owner, marks, int(e)):
            out[e] = 0
    return out


def final_marks(mesh: Mesh, rho, rho_solid: float, r_amr: float) -> np.ndarray:
    """Marks after both sweeps (Sec. 4, step 1)."""
    return sweep_balance(mesh, sweep_siblings(mesh, mark(mesh, rho, rho_solid, r_amr)))


def adapt(mesh: Mesh, marks, rho):
    """New (leaves, rho) after refinement, coarsening and 2:1 balancing."""
    L = mesh.L
    rho = np.asarray(rho, np.float64)
    index = leaf_index(mesh)
    out_leaves, out_rho = [], []
    done_parent = set()
    for e in range(mesh.Ne):
        lf = mesh.leaves[e]
        s = 1 << (L - int(lf[3]))
        if marks[e] == 1:
            h = s // 2
            for k in range(8):
                out_leaves.append([lf[0] + h * (k & 1), lf[1] + h * ((k >> 1) & 1), lf[2] + h * ((k >> 2) & 1),
                                   lf[3] + 1])
                out_rho.append(rho[e])
        elif marks[e] == -1:
            pa, ps = _parent(lf, L)
            key = (pa, int(lf[3]))
            if key in done_parent:
                continue
            done_parent.add(key)
            h = ps // 2
            kids = [index.get(((pa[0] + h * (k & 1), pa[1] + h * ((k >> 1) & 1), pa[2] + h * ((k >> 2) & 1)),
                               int(lf[3]))) for k in range(8)]
            if any(j is None or marks[j] != -1 for j in kids):
                raise ValueError("a family marked for derefinement is not 8 sibling leaves marked -1")
            total = 0.0
            for j in kids:            # sibling order (x fastest), one rounding per addition
                total += float(rho[j])
            out_leaves.append([pa[0], pa[1], pa[2], lf[3] - 1])
            out_rho.append(total / 8.0)
        else:
            out_leaves.append(list(lf))
            out_rho.append(rho[e])
    leaves = np.array(out_leaves, np.int64)
    rho_new = np.array(out_rho)
    # 2:1 balance: refine any leaf touching a leaf more than one level finer
    while True:
        owner = leaf_owner_map(mesh.nx, mesh.ny, mesh.nz, L, leaves)
        ext = np.array(owner.shape)
        need = np.zeros(leaves.shape[0], bool)
        for i, lf in enumerate(leaves):
            s = 1 << (L - int(lf[3]))
            lo = np.maximum(lf[:3] - 1, 0)
            hi = np.minimum(lf[:3] + s + 1, ext)
            nb = np.unique(owner[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
            if leaves[nb, 3].max() > lf[3] + 1:
                need[i] = True
        if not need.any():
            return leaves, rho_new
        nl, nr = [], []
        for i, lf in enumerate(leaves):
            if need[i]:
                h = (1 << (L - int(lf[3]))) // 2
                for k in range(8):
                    nl.append([lf[0] + h * (k & 1), lf[1] + h * ((k >> 1) & 1), lf[2] + h * ((k >> 2) & 1), lf[3] + 1])
                    nr.append(rho_new[i])
            else:
                nl.append(list(lf))
                nr.append(rho_new[i])
        leaves, rho_new = np.array(nl, np.int64), np.array(nr)


def rasterize(nx, ny, nz, L, leaves, rho) -> np.ndarray:
    owner = leaf_owner_map(nx, ny, nz, L, np.asarray(leaves, np.int64))
    return np.asarray(rho, np.float64)[owner]


def design_difference(nx, ny, nz, L, leaves1, rho1, leaves2, rho2) -> float:
    """Eq. 10 on the finest grid (cells of equal volume)."""
    a = rasterize(nx, ny, nz, L, leaves1, rho1)
    b = rasterize(nx, ny, nz, L, leaves2, rho2)
    return float(np.abs(a - b).sum() / a.sum())


def transfer_field(old: Mesh, u_full_old, points) -> np.ndarray:
    """(n, 3) values at integer finest-grid `points` (n, 3) of the old mesh's field u_full_old
    (3 Nn, hanging entries interpolated, i.e. C u)."""
    u = np.asarray(u_full_old, np.float64).reshape(-1, 3)
    owner = leaf_owner_map(old.nx, old.ny, old.nz, old.L, old.leaves)
    ext = np.array(owner.shape)
    pts = np.asarray(points, np.int64)
    cell = np.minimum(pts, ext - 1)                      # a cell whose closed box holds the point
    e = owner[cell[:, 0], cell[:, 1], cell[:, 2]]
    lf = old.leaves[e]
    s = (1 << (old.L - lf[:, 3])).astype(np.float64)
    t = (pts - lf[:, :3]) / s[:, None]                   # local coordinates in [0, 1]
    out = np.zeros((pts.shape[0], 3))
    for k in range(8):
        i, j, m_ = k & 1, (k >> 1) & 1, (k >> 2) & 1
        w = ((t[:, 0] if i else 1 - t[:, 0]) * (t[:, 1] if j else 1 - t[:, 1])
             * (t[:, 2] if m_ else 1 - t[:, 2]))
        out += w[:, None] * u[old.conn[e, k]]
    return out
