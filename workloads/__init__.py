"""Seeded synthetic inputs for the AMR topology-optimisation hot path.

This module builds the *inputs* that both the CUDA library and the oracle
consume: a 2:1-balanced list of octree leaves on a box, an element density
vector and nodal point loads.  It holds none of the method's arithmetic (no
node numbering, no constraints, no stiffness, no solver); the leaf list it
returns is checked independently by each consumer.

Geometry conventions (shared *input* format, not an implementation):

* The box is ``[0, 2] x [0, 1] x [0, 1]`` split into ``nx x ny x nz`` base
  cells of side ``h0 = 2 / nx`` (the 3D cantilever of the paper's Test 2 has
  the same 2:1:1 shape).
* ``L`` is the maximum refinement level.  Coordinates are integers on the
  finest grid, whose unit is ``h0 / 2**L``; a leaf at level ``l`` has side
  ``2**(L - l)`` units and an anchor (minimum corner) that is a multiple of it.
* A leaf is the int64 row ``(ix, iy, iz, level)``.

Recipes (seeded; the shapes follow the paper's 3D cantilever workloads):

* ``random_field_mesh`` -- a smoothed seeded N(0,1) field on the finest grid
  (three 3x3x3 box blurs, a logistic squash, then an affine map onto
  ``[rho_min, 1]``); leaves whose mean density lies in a band are refined, then
  the mesh is balanced.
* ``truss_mesh`` -- a seeded space truss (capsules around jittered members)
  standing in for a mid-optimisation cantilever design; leaves that meet the
  solid dilated by ``r_amr`` are refined to the finest level, as in the
  paper's refinement criterion (solid elements and a layer around them).
* ``batch_designs`` -- sixteen truss designs with two levels on bases of 2k x k x k cells
  (about 50k to 500k leaves), seeds 100-115, for batched solves.
* ``load_cases`` -- seeded load cases on the face x = 2 of a box (point loads and uniform face
  tractions at base-lattice points, which are nodes of every mesh of that box), for multi-load
  solves.
* ``unet_init`` -- seeded initial parameters of a network given by its parameter shapes.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy import ndimage

__all__ = [
    "Domain", "Workload", "uniform_leaves", "refine", "balance", "level_map",
    "smoothed_field", "random_field_mesh", "truss_mesh", "config1", "config1b",
    "config2", "small_truss", "load_at", "batch_designs", "unet_init", "load_cases",
]


@dataclasses.dataclass(frozen=True)
class Domain:
    nx: int
    ny: int
    nz: int
    L: int
    h0: float

    @property
    def fine_shape(self):
        s = 1 << self.L
        return (self.nx * s, self.ny * s, self.nz * s)

    @property
    def h_min(self):
        return self.h0 / (1 << self.L)


@dataclasses.dataclass
class Workload:
    name: str
    dom: Domain
    leaves: np.ndarray          # (Ne, 4) int64: ix, iy, iz, level
    rho: np.ndarray             # (Ne,) float64, same order as ``leaves``
    load_nodes: np.ndarray      # (nl, 3) int64 finest-grid node coordinates
    load_comp: np.ndarray       # (nl,) int64 component 0/1/2
    load_val: np.ndarray        # (nl,) float64
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    penal: float = 3.0
    rho_min: float = 1e-3
    dirichlet_faces: int = 1    # bit 0: x = 0 clamped

    @property
    def r_min(self):
        return 1.5 * self.dom.h_min


def uniform_leaves(dom: Domain) -> np.ndarray:
    s = 1 << dom.L
    ix, iy, iz = np.meshgrid(np.arange(dom.nx), np.arange(dom.ny), np.arange(dom.nz), indexing="ij")
    out = np.stack([ix.ravel() * s, iy.ravel() * s, iz.ravel() * s, np.zeros(ix.size, np.int64)], axis=1)
    return out.astype(np.int64)


def refine(dom: Domain, leaves: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Split every masked leaf into its 8 children."""
    mask = np.asarray(mask, bool) & (leaves[:, 3] < dom.L)
    keep = leaves[~mask]
    par = leaves[mask]
    if par.shape[0] == 0:
        return keep.copy()
    half = (1 << (dom.L - par[:, 3] - 1)).astype(np.int64)
    kids = []
    for c in range(8):
        dx, dy, dz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        kids.append(np.stack([par[:, 0] + dx * half, par[:, 1] + dy * half, par[:, 2] + dz * half,
                              par[:, 3] + 1], axis=1))
    return np.concatenate([keep] + kids, axis=0)


def level_map(dom: Domain, leaves: np.ndarray) -> np.ndarray:
    """Dense finest-grid array holding the level of the leaf covering each cell."""
    out = np.full(dom.fine_shape, -1, np.int8)
    for lvl in range(dom.L + 1):
        sel = leaves[leaves[:, 3] == lvl]
        s = 1 << (dom.L - lvl)
        coarse = np.full((dom.fine_shape[0] // s, dom.fine_shape[1] // s, dom.fine_shape[2] // s), -1, np.int8)
        coarse[sel[:, 0] // s, sel[:, 1] // s, sel[:, 2] // s] = lvl
        up = np.repeat(np.repeat(np.repeat(coarse, s, 0), s, 1), s, 2)
        np.copyto(out, up, where=up >= 0)
    return out


def _block_reduce_max(a: np.ndarray, s: int) -> np.ndarray:
    X, Y, Z = a.shape
    return a.reshape(X // s, s, Y // s, s, Z // s, s).max(axis=(1, 3, 5))


def balance(dom: Domain, leaves: np.ndarray) -> np.ndarray:
    """Refine leaves until any two leaves that touch (even at one point) differ
    by at most one level -- the "level-one incompatibility" the paper allows."""
    while True:
        lv = level_map(dom, leaves)
        if (lv < 0).any():
            raise ValueError("leaves do not cover the domain")
        nb = ndimage.maximum_filter(lv, size=3, mode="nearest")
        need = np.zeros(leaves.shape[0], bool)
        for lvl in range(dom.L + 1):
            idx = np.nonzero(leaves[:, 3] == lvl)[0]
            if idx.size == 0:
                continue
            s = 1 << (dom.L - lvl)
            bm = _block_reduce_max(nb, s)
            sel = leaves[idx]
            need[idx] = bm[sel[:, 0] // s, sel[:, 1] // s, sel[:, 2] // s] > lvl + 1
        if not need.any():
            return leaves
        leaves = refine(dom, leaves, need)


def smoothed_field(shape, seed: int, passes: int = 3, lo: float = 1e-3, hi: float = 1.0,
                   slope: float = 6.0) -> np.ndarray:
    """N(0,1) i.i.d. values, ``passes`` 3x3x3 box blurs (edge replicated), standardised, passed
    through a logistic of the given slope (so that most cells sit near 0 or 1, as in a SIMP
    design, with intermediate values along interfaces) and mapped affinely onto [lo, hi]."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape)
    for _ in range(passes):
        a = ndimage.uniform_filter(a, size=3, mode="nearest")
    a = (a - a.mean()) / a.std()
    a = 1.0 / (1.0 + np.exp(-slope * a))
    a = (a - a.min()) / (a.max() - a.min())
    return lo + (hi - lo) * a


def _leaf_mean(dom: Domain, leaves: np.ndarray, field: np.ndarray) -> np.ndarray:
    out = np.empty(leaves.shape[0])
    for lvl in range(dom.L + 1):
        idx = np.nonzero(leaves[:, 3] == lvl)[0]
        if idx.size == 0:
            continue
        s = 1 << (dom.L - lvl)
        X, Y, Z = field.shape
        bm = field.reshape(X // s, s, Y // s, s, Z // s, s).mean(axis=(1, 3, 5))
        sel = leaves[idx]
        out[idx] = bm[sel[:, 0] // s, sel[:, 1] // s, sel[:, 2] // s]
    return out


def load_at(dom: Domain, x: float, y: float, z: float, comp: int = 2, val: float = -1.0):
    u = dom.h_min
    node = np.array([[round(x / u), round(y / u), round(z / u)]], np.int64)
    return node, np.array([comp], np.int64), np.array([val], np.float64)


def random_field_mesh(name, dom: Domain, seed: int, bands, rho_min=1e-3) -> Workload:
    """Refine leaves of level ``l`` whose mean field value lies in ``bands[l]``."""
    field = smoothed_field(dom.fine_shape, seed, lo=rho_min)
    leaves = uniform_leaves(dom)
    for lvl in range(dom.L):
        lo, hi = bands[min(lvl, len(bands) - 1)]
        m = _leaf_mean(dom, leaves, field)
        leaves = refine(dom, leaves, (leaves[:, 3] == lvl) & (m > lo) & (m < hi))
    leaves = balance(dom, leaves)
    rho = _leaf_mean(dom, leaves, field)
    ln, lc, lv = load_at(dom, 2.0, 0.5, 0.5)
    return Workload(name, dom, leaves, rho, ln, lc, lv, rho_min=rho_min)


def config1(seed: int = 1) -> Workload:
    """Base 8x4x4, one level; base cells with mean density in (0.1, 0.9) are refined."""
    return random_field_mesh("cantilever_8x4x4_L1", Domain(8, 4, 4, 1, 0.25), seed, [(0.1, 0.9)])


def config1b(seed: int = 1) -> Workload:
    """Base 8x4x4, two levels (about 1-3k elements)."""
    return random_field_mesh("cantilever_8x4x4_L2", Domain(8, 4, 4, 2, 0.25), seed, [(0.1, 0.9), (0.4, 0.6)])


# ---------------------------------------------------------------- truss recipe
def _truss_members(rng, jitter):
    """Jittered nodes of a tapered four-chord space truss from x = 0 to the tip (2, .5, .5)."""
    xs = [0.0, 0.5, 1.0, 1.5]
    nodes = []
    for x in xs:
        w = 0.36 * (1.0 - x / 2.3) + 0.04
        for sy, sz in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
            p = np.array([x, 0.5 + sy * w, 0.5 + sz * w])
            if x > 0:
                p = p + rng.uniform(-jitter, jitter, 3)
            nodes.append(p)
    nodes.append(np.array([2.0, 0.5, 0.5]))
    nodes = np.array(nodes)
    tip = len(nodes) - 1
    mem = []
    for b in range(len(xs)):
        base = 4 * b
        for k in range(4):
            a = base + k
            if b + 1 < len(xs):
                mem.append((a, a + 4))                  # chord
                mem.append((a, base + 4 + (k + 1) % 4))  # face diagonal
            else:
                mem.append((a, tip))                    # converge on the loaded tip
            if b > 0:
                mem.append((a, base + (k + 1) % 4))     # ring
    return nodes, np.array(mem)


def _capsule_sdf(pts, a, b, r):
    ab = b - a
    t = np.clip(((pts - a) @ ab) / (ab @ ab), 0.0, 1.0)
    d = np.linalg.norm(pts - (a + t[:, None] * ab), axis=1)
    return d - r


def truss_sdf(pts, seed: int, r0: float, jitter: float = 0.03):
    rng = np.random.default_rng(seed)
    nodes, mem = _truss_members(rng, jitter)
    radii = r0 * (1.0 + 0.25 * rng.uniform(-1, 1, len(mem)))
    phi = np.full(pts.shape[0], np.inf)
    for (i, j), r in zip(mem, radii):
        phi = np.minimum(phi, _capsule_sdf(pts, nodes[i], nodes[j], r))
    return phi


def _centres(dom: Domain, leaves):
    s = (1 << (dom.L - leaves[:, 3])).astype(np.float64)
    return (leaves[:, :3] + 0.5 * s[:, None]) * dom.h_min


def truss_mesh(name, dom: Domain, seed: int, r0: float, r_amr_cells: float = 2.0, rho_min=1e-3) -> Workload:
    """Leaves meeting the truss dilated by ``r_amr`` are refined level by level, then balanced."""
    leaves = uniform_leaves(dom)
    r_amr = r_amr_cells * dom.h_min
    for lvl in range(dom.L):
        sel = leaves[:, 3] == lvl
        c = _centres(dom, leaves[sel])
        h = dom.h0 / (1 << lvl)
        phi = truss_sdf(c, seed, r0)
        m = np.zeros(leaves.shape[0], bool)
        m[np.nonzero(sel)[0]] = phi < r_amr + 0.5 * np.sqrt(3.0) * h
        leaves = refine(dom, leaves, m)
    leaves = balance(dom, leaves)
    phi = truss_sdf(_centres(dom, leaves), seed, r0)
    heav = np.clip(0.5 - phi / (2.0 * dom.h_min), 0.0, 1.0)
    rho = rho_min + (1.0 - rho_min) * heav
    ln, lc, lv = load_at(dom, 2.0, 0.5, 0.5)
    return Workload(name, dom, leaves, rho, ln, lc, lv, rho_min=rho_min)


def config2(seed: int = 2) -> Workload:
    """Base 48x24x24, three levels along a seeded truss interface (about 1-2M leaves)."""
    return truss_mesh("cantilever_48x24x24_L3_truss", Domain(48, 24, 24, 3, 2.0 / 48), seed, r0=0.045)


def small_truss(seed: int = 2, base=(12, 6, 6), L: int = 2, r0: float = 0.06) -> Workload:
    """The config-2 recipe on a coarser base: sizes the oracle's direct solver handles in seconds."""
    nx, ny, nz = base
    return truss_mesh(f"cantilever_{nx}x{ny}x{nz}_L{L}_truss", Domain(nx, ny, nz, L, 2.0 / nx), seed, r0=r0)


def batch_designs(n: int = 16, seed0: int = 100):
    """Independent designs for batched solves: the truss recipe with two levels on bases of
    2k x k x k cells, k stepping from 9 to 26 across the batch (about 50k to 500k leaves),
    seeds seed0, seed0 + 1, ..."""
    ks = np.linspace(9, 26, n).round().astype(int)
    return [truss_mesh(f"cantilever_{2 * k}x{k}x{k}_L2_truss_s{seed0 + i}", Domain(2 * k, k, k, 2, 1.0 / k),
                       seed0 + i, r0=0.045) for i, k in enumerate(ks)]


def load_cases(dom: Domain, n: int = 8, seed0: int = 10):
    """n load cases [(node_xyz (k, 3), comp (k,), val (k,))] with seeds seed0, seed0 + 1, ...:
    even cases a unit point load at a random base-lattice point of the face x = 2 in a random
    direction and sign; odd cases a uniform traction of total -1 in a random direction over all
    base-lattice points of that face (corner, edge and interior points weighted 1/4, 1/2, 1)."""
    s = 1 << dom.L
    X = dom.nx * s
    jj, kk = np.meshgrid(np.arange(dom.ny + 1) * s, np.arange(dom.nz + 1) * s, indexing="ij")
    face = np.stack([np.full(jj.size, X), jj.ravel(), kk.ravel()], 1).astype(np.int64)
    wy = np.where((jj.ravel() == 0) | (jj.ravel() == dom.ny * s), 0.5, 1.0)
    wz = np.where((kk.ravel() == 0) | (kk.ravel() == dom.nz * s), 0.5, 1.0)
    w = wy * wz
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        comp = int(rng.integers(3))
        if i % 2 == 0:
            p = face[rng.integers(len(face))][None]
            out.append((p, np.array([comp]), np.array([float(rng.choice([-1.0, 1.0]))])))
        else:
            out.append((face, np.full(len(face), comp), -w / w.sum()))
    return out


def unet_init(shapes, seed: int = 0):
    """Seeded initial parameters for a network given as [(name, shape)]: weights normal with
    variance 2 / fan_in (fan_in = input channels x kernel volume), biases uniform in +-0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in shapes:
        if len(shape) > 1:
            fan_in = int(np.prod(shape[1:]))
            out.append(rng.standard_normal(shape) * np.sqrt(2.0 / fan_in))
        else:
            out.append(rng.uniform(-0.1, 0.1, shape))
    return out
