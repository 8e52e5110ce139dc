"""Oracle mesh tables for a 2:1-balanced octree hex mesh (paper Sec. 4 and 6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions (paper Sec. 6, "level-one mesh incompatibility" and Eq. 6):

* A *leaf* ``(ix, iy, iz, l)`` is the closed box ``[a, a + s]`` with anchor
  ``a = (ix, iy, iz)`` and side ``s = 2**(L - l)`` finest-grid units.
* The *nodes* are the distinct leaf corners.
* A node is *hanging* iff it lies in the relative interior of an edge or a face
  of some leaf.  Its value is the linear (edge) or bilinear (face) interpolation
  of that edge's / face's corner values -- the "linear interpolation from
  unconstrained DOFs" of Sec. 6.  Masters that are themselves hanging are
  substituted recursively (none occur on a balanced mesh; this is asserted).
* Balance ("level-one incompatibility"): any two leaves whose closures meet,
  even in a single point, differ by at most one level.

Canonical orders (a reading: the paper is silent):

* elements are sorted by the Morton key of their anchor;
* nodes are sorted by the Morton key of their integer coordinates;
* the Morton key interleaves bit ``i`` of x, y, z at bits ``3i``, ``3i+1``,
  ``3i+2``;
* local corner ``k = i + 2 j + 4 m`` sits at ``a + s * (i, j, m)``.
"""
from __future__ import annotations

import dataclasses
from fractions import Fraction

import numpy as np


def morton_key(x, y, z) -> np.ndarray:
    """Bit interleave, written bit by bit (21 bits per axis)."""
    x = np.asarray(x, np.uint64)
    y = np.asarray(y, np.uint64)
    z = np.asarray(z, np.uint64)
    key = np.zeros(np.broadcast(x, y, z).shape, np.uint64)
    one = np.uint64(1)
    for b in range(21):
        bb = np.uint64(b)
        key |= ((x >> bb) & one) << np.uint64(3 * b)
        key |= ((y >> bb) & one) << np.uint64(3 * b + 1)
        key |= ((z >> bb) & one) << np.uint64(3 * b + 2)
    return key


CORNER_OFFSETS = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], np.int64)


@dataclasses.dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    L: int
    h0: float
    leaves: np.ndarray        # (Ne, 4) canonical order
    perm: np.ndarray          # canonical element i is input leaf perm[i]
    nodes: np.ndarray         # (Nn, 3) integer coordinates, canonical order
    conn: np.ndarray          # (Ne, 8) node ids
    hanging: dict             # node id -> list of (master node id, Fraction weight), masters ascending
    dirichlet: np.ndarray     # (Nn,) bool

    @property
    def Ne(self):
        return self.leaves.shape[0]

    @property
    def Nn(self):
        return self.nodes.shape[0]

    @property
    def size(self):
        """Element side in finest-grid units."""
        return (1 << (self.L - self.leaves[:, 3])).astype(np.int64)

    @property
    def h(self):
        """Element side length."""
        return self.size * (self.h0 / (1 << self.L))

    @property
    def volume(self):
        return self.h ** 3

    @property
    def centres(self):
        u = self.h0 / (1 << self.L)
        return (self.leaves[:, :3] + 0.5 * self.size[:, None]) * u

    @property
    def fine_shape(self):
        s = 1 << self.L
        return (self.nx * s, self.ny * s, self.nz * s)

    def hanging_ids(self):
        return np.array(sorted(self.hanging), np.int64)


def check_leaves(nx, ny, nz, L, leaves) -> None:
    """Reject leaves that are out of range, misaligned, overlapping or not covering."""
    leaves = np.asarray(leaves, np.int64)
    if leaves.ndim != 2 or leaves.shape[1] != 4 or leaves.shape[0] == 0:
        raise ValueError("leaves must be a non-empty (n, 4) array")
    lvl = leaves[:, 3]
    if (lvl < 0).any() or (lvl > L).any():
        raise ValueError("leaf level out of range")
    s = (1 << (L - lvl)).astype(np.int64)
    ext = np.array([nx, ny, nz], np.int64) << L
    a = leaves[:, :3]
    if (a < 0).any() or ((a + s[:, None]) > ext).any():
        raise ValueError("leaf outside the domain")
    if ((a % s[:, None]) != 0).any():
        raise ValueError("leaf anchor not aligned to its size")
    # every finest cell covered exactly once
    count = np.zeros(tuple(ext), np.int32)
    for lv in np.unique(lvl):
        sel = a[lvl == lv]
        sz = int(1 << (L - lv))
        for dx in range(sz):
            for dy in range(sz):
                for dz in range(sz):
                    np.add.at(count, (sel[:, 0] + dx, sel[:, 1] + dy, sel[:, 2] + dz), 1)
    if (count != 1).any():
        raise ValueError("leaves overlap or leave gaps")


def leaf_owner_map(nx, ny, nz, L, leaves) -> np.ndarray:
    """Finest-grid cell -> index of the leaf containing it (leaves assumed valid)."""
    ext = (nx << L, ny << L, nz << L)
    owner = np.full(ext, -1, np.int64)
    lvl = leaves[:, 3]
    for lv in np.unique(lvl):
        idx = np.nonzero(lvl == lv)[0]
        sel = leaves[idx]
        sz = int(1 << (L - lv))
        for dx in range(sz):
            for dy in range(sz):
                for dz in range(sz):
                    owner[sel[:, 0] + dx, sel[:, 1] + dy, sel[:, 2] + dz] = idx
    return owner


def _closure_leaves(owner, pts):
    """For each point, the (up to 8) leaves whose closed box contains it; -1 pads."""
    ext = np.array(owner.shape)
    out = np.full((pts.shape[0], 8), -1, np.int64)
    for k, off in enumerate(CORNER_OFFSETS):
        c = pts - 1 + off
        ok = ((c >= 0) & (c < ext)).all(axis=1)
        out[ok, k] = owner[c[ok, 0], c[ok, 1], c[ok, 2]]
    return out


def check_balance(nx, ny, nz, L, leaves) -> None:
    """Every node's closure-leaves differ by at most one level (paper Sec. 6)."""
    owner = leaf_owner_map(nx, ny, nz, L, leaves)
    s = (1 << (L - leaves[:, 3])).astype(np.int64)
    corners = (leaves[:, None, :3] + CORNER_OFFSETS[None] * s[:, None, None]).reshape(-1, 3)
    pts = np.unique(corners, axis=0)
    cl = _closure_leaves(owner, pts)
    lv = np.where(cl >= 0, leaves[np.maximum(cl, 0), 3], -1)
    hi = lv.max(axis=1)
    lo = np.where(cl >= 0, lv, 1 << 30).min(axis=1)
    if (hi - lo > 1).any():
        raise ValueError("mesh is not 2:1 balanced")


def _point_in_leaf(p, leaf, L):
    """Relation of integer point p to the closed box of ``leaf``: returns the list of axes along
    which p is strictly inside (0 axes: corner, 1: edge interior, 2: face interior)."""
    s = 1 << (L - int(leaf[3]))
    inside = []
    for ax in range(3):
        lo = int(leaf[ax])
        if p[ax] < lo or p[ax] > lo + s:
            return None
        if lo < p[ax] < lo + s:
            inside.append(ax)
    return inside


def _interp_masters(p, leaf, L, inside):
    """Corner points of the edge/face of ``leaf`` through p and their (bi)linear weights."""
    s = 1 << (L - int(leaf[3]))
    out = []
    combos = [[]]
    for ax in inside:
        combos = [c + [(ax, side)] for c in combos for side in (0, 1)]
    for c in combos:
        q = list(p)
        w = Fraction(1)
        for ax, side in c:
            lo = int(leaf[ax])
            q[ax] = lo + side * s
            t = Fraction(p[ax] - lo, s)
            w *= t if side else (1 - t)
        out.append((tuple(q), w))
    return out


def build_mesh(nx, ny, nz, L, h0, leaves, dirichlet_faces=1, validate=True) -> Mesh:
    """Canonical tables for a leaf set (paper Sec. 6)."""
    leaves = np.asarray(leaves, np.int64)
    if validate:
        check_leaves(nx, ny, nz, L, leaves)
        check_balance(nx, ny, nz, L, leaves)
    key = morton_key(leaves[:, 0], leaves[:, 1], leaves[:, 2])
    perm = np.argsort(key, kind="stable")
    leaves = leaves[perm]
    s = (1 << (L - leaves[:, 3])).astype(np.int64)
    corners = leaves[:, None, :3] + CORNER_OFFSETS[None] * s[:, None, None]      # (Ne, 8, 3)
    flat = corners.reshape(-1, 3)
    nkey = morton_key(flat[:, 0], flat[:, 1], flat[:, 2])
    ukey, first, inv = np.unique(nkey, return_index=True, return_inverse=True)
    nodes = flat[first]
    conn = inv.reshape(-1, 8).astype(np.int64)
    node_of = {tuple(p): i for i, p in enumerate(map(tuple, nodes))}

    owner = leaf_owner_map(nx, ny, nz, L, leaves)
    cl = _closure_leaves(owner, nodes)                                # (Nn, 8)
    valid = cl >= 0
    lf = leaves[np.maximum(cl, 0)]                                    # (Nn, 8, 4)
    sz = (1 << (L - lf[..., 3])).astype(np.int64)
    lo = lf[..., :3]
    p = nodes[:, None, :]
    strictly = (p > lo) & (p < lo + sz[..., None])                    # (Nn, 8, 3)
    n_in = strictly.sum(axis=2)
    if (valid & (n_in == 3)).any():
        raise ValueError("node strictly inside a leaf: overlapping leaves")
    cand = valid & (n_in > 0)
    # the coarsest leaf having the node inside an edge or face decides the interpolation
    score = np.where(cand, sz, -1)
    pick = score.argmax(axis=1)
    is_h = score.max(axis=1) > 0
    raw = {}
    for i in np.nonzero(is_h)[0]:
        e = int(cl[i, pick[i]])
        pt = tuple(int(v) for v in nodes[i])
        inside = [ax for ax in range(3) if strictly[i, pick[i], ax]]
        raw[int(i)] = [(node_of[q], w) for q, w in _interp_masters(pt, leaves[e], L, inside)]

    def resolve(i, depth=0):
        if depth > 64:
            raise ValueError("constraint chain does not terminate")
        acc = {}
        for m, w in raw[i]:
            if m in raw:
                for mm, ww in resolve(m, depth + 1):
                    acc[mm] = acc.get(mm, Fraction(0)) + w * ww
            else:
                acc[m] = acc.get(m, Fraction(0)) + w
        return sorted(acc.items())

    hanging = {}
    chains = False
    for i in raw:
        if any(m in raw for m, _ in raw[i]):
            chains = True
        hanging[i] = [(m, w) for m, w in resolve(i) if w != 0]
    if validate and chains:
        raise AssertionError("constraint chain on a balanced mesh")

    ext = np.array([nx, ny, nz], np.int64) << L
    dmask = np.zeros(nodes.shape[0], bool)
    for f in range(6):
        if dirichlet_faces >> f & 1:
            ax, side = f // 2, f % 2
            dmask |= nodes[:, ax] == (ext[ax] if side else 0)
    return Mesh(nx, ny, nz, L, float(h0), leaves, perm, nodes, conn, hanging, dmask)


def hanging_bruteforce(nx, ny, nz, L, leaves):
    """O(Nn * Ne) restatement of the hanging definition, for tiny meshes: every node against
    every leaf.  Returns {node coordinate: sorted [(master coordinate, weight)]} without chains."""
    leaves = np.asarray(leaves, np.int64)
    pts = set()
    for lf in leaves:
        s = 1 << (L - int(lf[3]))
        for off in CORNER_OFFSETS:
            pts.add(tuple(int(v) for v in lf[:3] + s * off))
    out = {}
    for p in sorted(pts):
        best = None
        for lf in leaves:
            ins = _point_in_leaf(p, lf, L)
            if ins is None or len(ins) == 0:
                continue
            s = 1 << (L - int(lf[3]))
            if best is None or s > best[0]:
                best = (s, lf, ins)
        if best is not None:
            out[p] = sorted(_interp_masters(p, best[1], L, best[2]))
    return out
