"""Pins for the adaptation oracle (paper Sec. 4, balancing of Sec. 6) and the design
difference of Eq. 10: hand-worked meshes, brute force, closed forms and invariants."""
import numpy as np
import pytest

import workloads as W
from oracle import amr as A
from oracle import mesh as M


def _mesh(dom, leaves):
    return M.build_mesh(dom.nx, dom.ny, dom.nz, dom.L, dom.h0, np.asarray(leaves, np.int64))


def _children(anchor, level, L):
    h = 1 << (L - level - 1)
    return [[anchor[0] + h * (k & 1), anchor[1] + h * ((k >> 1) & 1), anchor[2] + h * ((k >> 2) & 1), level + 1]
            for k in range(8)]


def _by_anchor(mesh, values):
    return {(tuple(int(v) for v in lf[:3]), int(lf[3])): values[i] for i, lf in enumerate(mesh.leaves)}


# ---------------------------------------------------------------- hand-worked cases
def test_hand_case_refine_and_balance():
    """2x1x1 box, L = 2, h0 = 1.  Cell A (x < 1) split into 8 children, cell B whole.
    One solid child at the origin, r_AMR = 0.6: its three face neighbours (centre distance
    0.5) refine, the other four children (0.707, 0.866) are void but their family is not all
    -1, and B (level 0) cannot coarsen.  Refining child 1 (touching B at x = 1) puts level 2
    against level 0, so balancing splits B: 4 x 8 + 4 + 8 = 44 leaves."""
    dom = W.Domain(2, 1, 1, 2, 1.0)
    leaves = _children((0, 0, 0), 0, 2) + [[4, 0, 0, 0]]
    m = _mesh(dom, leaves)
    rho_in = {(0, 0, 0, 1): 1.0}
    rho = np.array([rho_in.get(tuple(int(v) for v in lf), 0.01) for lf in m.leaves])
    raw = A.mark(m, rho, 0.5, 0.6)
    got = _by_anchor(m, raw)
    want_plus = {(0, 0, 0), (2, 0, 0), (0, 2, 0), (0, 0, 2)}
    for (a, lvl), v in got.items():
        if lvl == 0:
            assert v == 0
        else:
            assert v == (1 if a in want_plus else -1), (a, v)
    # centres exactly r apart are not below r: at r = 0.5 only the solid child refines
    tie = _by_anchor(m, A.mark(m, rho, 0.5, 0.5))
    assert [v for (a, lvl), v in tie.items() if lvl == 1].count(1) == 1
    assert tie[((0, 0, 0), 1)] == 1 and tie[((2, 0, 0), 1)] == -1
    fin = A.final_marks(m, rho, 0.5, 0.6)
    for (a, lvl), v in _by_anchor(m, fin).items():
        assert v == (1 if lvl == 1 and a in want_plus else 0)
    leaves2, rho2 = A.adapt(m, fin, rho)
    assert leaves2.shape[0] == 44
    lv = leaves2[:, 3]
    assert (lv == 2).sum() == 32 and (lv == 1).sum() == 12 and (lv == 0).sum() == 0
    M.check_leaves(2, 1, 1, 2, leaves2)
    M.check_balance(2, 1, 1, 2, leaves2)
    # children inherit: the 8 children of the solid element carry 1, B's children carry 0.01
    solid = (leaves2[:, 0] < 2) & (leaves2[:, 1] < 2) & (leaves2[:, 2] < 2)
    assert (rho2[solid] == 1.0).all() and solid.sum() == 8
    assert (rho2[leaves2[:, 0] >= 4] == 0.01).all()


def _three_level_case(solid_touches_family: bool):
    """2x1x1 box, L = 3, h0 = 1.  A = [0,1] and B = [1,2] split into level-1 children; A's child
    A1 (x in [.5, 1], y, z < .5) and B's child B0 (x in [1, 1.5], y, z < .5) split again into
    level-2 children.  One level-2 child of B0 is solid: the one at the x = 1 face (touching
    A1) or the one at the far corner x in [1.25, 1.5], y, z in [.25, .5]."""
    L = 3
    leaves = []
    for k, c in enumerate(_children((0, 0, 0), 0, L)):
        leaves += _children(c[:3], 1, L) if k == 1 else [c]
    for k, c in enumerate(_children((8, 0, 0), 0, L)):
        leaves += _children(c[:3], 1, L) if k == 0 else [c]
    dom = W.Domain(2, 1, 1, L, 1.0)
    m = _mesh(dom, leaves)
    solid_anchor = (8, 0, 0) if solid_touches_family else (10, 2, 2)
    rho = np.array([1.0 if (tuple(int(v) for v in lf[:3]) == solid_anchor and lf[3] == 2) else 0.01
                    for lf in m.leaves])
    return dom, m, rho


def test_hand_case_incompatibility_sweep_blocks_coarsening():
    """The solid level-2 child touching A1 refines to level 3, so coarsening A1's children
    to level 1 would put level 1 against level 3: the second sweep must veto it."""
    dom, m, rho = _three_level_case(True)
    raw = A.mark(m, rho, 0.5, 0.1)
    s1 = A.sweep_siblings(m, raw)
    fam = (m.leaves[:, 0] >= 4) & (m.leaves[:, 0] < 8) & (m.leaves[:, 1] < 4) & (m.leaves[:, 2] < 4)
    assert fam.sum() == 8 and (s1[fam] == -1).all()           # sweep 1 keeps A1's family
    assert (s1[~fam] <= 0).sum() == m.Ne - 8 - 1                # everything else 0 but the solid one
    fin = A.sweep_balance(m, s1)
    assert (fin[fam] == 0).all()                                # sweep 2 vetoes it
    assert (fin == 1).sum() == 1 and (fin == -1).sum() == 0
    leaves2, rho2 = A.adapt(m, fin, rho)
    assert leaves2.shape[0] == m.Ne - 1 + 8
    M.check_balance(2, 1, 1, 3, leaves2)


def test_hand_case_family_coarsens_when_compatible():
    """Same mesh with the solid element at B0's far corner: nothing touching A1 ends finer
    than level 2, so A1's family merges (rho = mean).  The solid element's 8 level-3 children
    touch all 7 level-1 children of B (faces at x = 1.5, y = .5, z = .5, their edges and the
    corner), which balancing splits: 30 - 8 + 1 - 1 + 8 - 7 + 56 = 79 leaves, of which 8 at
    level 3, 7 + 56 at level 2 and 7 + 1 at level 1."""
    dom, m, rho = _three_level_case(False)
    fin = A.final_marks(m, rho, 0.5, 0.1)
    fam = (m.leaves[:, 0] >= 4) & (m.leaves[:, 0] < 8) & (m.leaves[:, 1] < 4) & (m.leaves[:, 2] < 4)
    assert (fin[fam] == -1).all() and (fin == -1).sum() == 8 and (fin == 1).sum() == 1
    leaves2, rho2 = A.adapt(m, fin, rho)
    assert leaves2.shape[0] == 79
    assert np.bincount(leaves2[:, 3], minlength=4).tolist() == [0, 8, 63, 8]
    M.check_leaves(2, 1, 1, 3, leaves2)
    M.check_balance(2, 1, 1, 3, leaves2)
    parent = (leaves2[:, 0] == 4) & (leaves2[:, 1] == 0) & (leaves2[:, 2] == 0) & (leaves2[:, 3] == 1)
    assert parent.sum() == 1 and rho2[parent][0] == pytest.approx(0.01, rel=1e-15)


# ---------------------------------------------------------------- brute force and invariants
def _moved_design(w, m, seed):
    """A design that no longer matches the mesh: a thicker truss of another seed sampled at
    the element centres (solid material on coarse elements, void on fine ones)."""
    phi = W.truss_sdf(m.centres, seed, r0=0.09)
    return np.clip(0.5 - phi / (2.0 * w.dom.h_min), 1e-3, 1.0)


@pytest.mark.parametrize("seed,r_cells", [(1, 1.3), (3, 2.0), (5, 3.7), (2, 1.0)])
def test_mark_matches_bruteforce(seed, r_cells):
    w = W.config1b(seed)
    m = _mesh(w.dom, w.leaves)
    rho = w.rho[m.perm]
    r = r_cells * w.dom.h_min
    np.testing.assert_array_equal(A.mark(m, rho, 0.5, r), A.mark_bruteforce(m, rho, 0.5, r))


def _brute_marks_after_sweeps(m, raw):
    """Sweeps written from scratch on a dense level/owner grid, no shared helpers."""
    L = m.L
    ext = np.array(m.fine_shape)
    owner = -np.ones(tuple(ext), np.int64)
    for i, lf in enumerate(m.leaves):
        s = 1 << (L - int(lf[3]))
        owner[lf[0]:lf[0] + s, lf[1]:lf[1] + s, lf[2]:lf[2] + s] = i
    out = raw.copy()
    for e in range(m.Ne):
        if raw[e] != -1:
            continue
        lf = m.leaves[e]
        s = 1 << (L - int(lf[3]))
        p = (lf[:3] // (2 * s)) * (2 * s)
        block = owner[p[0]:p[0] + 2 * s, p[1]:p[1] + 2 * s, p[2]:p[2] + 2 * s]
        kids = np.unique(block)
        ok = kids.size == 8 and all(m.leaves[k, 3] == lf[3] and raw[k] == -1 for k in kids)
        if ok:
            lo = np.maximum(p - 1, 0)
            hi = np.minimum(p + 2 * s + 1, ext)
            for d in np.unique(owner[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]):
                if m.leaves[d, 3] + (raw[d] == 1) > lf[3]:
                    ok = False
        if not ok:
            out[e] = 0
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_sweeps_match_bruteforce_and_keep_balance(seed):
    w = W.config1b(seed)
    m = _mesh(w.dom, w.leaves)
    rho = _moved_design(w, m, seed + 7)
    r = 1.6 * w.dom.h_min
    raw = A.mark(m, rho, 0.5, r)
    fin = A.final_marks(m, rho, 0.5, r)
    np.testing.assert_array_equal(fin, _brute_marks_after_sweeps(m, raw))
    assert (fin == -1).any() and (fin == 1).any()
    # refine +1 and merge -1 families without the balancing step: no merged parent may sit
    # next to a leaf more than one level finer (the purpose of the second sweep)
    d = w.dom
    L = d.L
    pre = []
    merged = set()
    for e in range(m.Ne):
        lf = m.leaves[e]
        s = 1 << (L - int(lf[3]))
        if fin[e] == 1:
            pre += _children(lf[:3], int(lf[3]), L)
        elif fin[e] == -1:
            p = tuple(int(v) // (2 * s) * (2 * s) for v in lf[:3])
            if p not in merged:
                merged.add(p)
                pre.append([p[0], p[1], p[2], int(lf[3]) - 1])
        else:
            pre.append(list(lf))
    pre = np.array(pre, np.int64)
    M.check_leaves(d.nx, d.ny, d.nz, L, pre)
    own = M.leaf_owner_map(d.nx, d.ny, d.nz, L, pre)
    ext = np.array(own.shape)
    for i, lf in enumerate(pre):
        if (tuple(int(v) for v in lf[:3])) not in merged:
            continue
        s = 1 << (L - int(lf[3]))
        lo = np.maximum(lf[:3] - 1, 0)
        hi = np.minimum(lf[:3] + s + 1, ext)
        assert pre[np.unique(own[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]), 3].max() <= lf[3] + 1


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_adapt_tiles_balances_and_conserves_mass(seed):
    w = W.config1b(seed)
    d = w.dom
    m = _mesh(d, w.leaves)
    rho = _moved_design(w, m, seed + 7)
    fin = A.final_marks(m, rho, 0.5, 1.6 * d.h_min)
    assert (fin == -1).any() and (fin == 1).any()
    leaves2, rho2 = A.adapt(m, fin, rho)
    M.check_leaves(d.nx, d.ny, d.nz, d.L, leaves2)
    M.check_balance(d.nx, d.ny, d.nz, d.L, leaves2)
    v1 = (1 << (d.L - m.leaves[:, 3])).astype(np.float64) ** 3
    v2 = (1 << (d.L - leaves2[:, 3])).astype(np.float64) ** 3
    assert np.sum(rho2 * v2) == pytest.approx(np.sum(rho * v1), rel=1e-13)
    # Morton order is kept (children in place of their parent, parents in place of the family)
    m2 = _mesh(d, leaves2)
    np.testing.assert_array_equal(m2.perm, np.arange(leaves2.shape[0]))
    # outside merged families every finest cell keeps its density exactly (children inherit)
    old = A.rasterize(d.nx, d.ny, d.nz, d.L, m.leaves, rho)
    new = A.rasterize(d.nx, d.ny, d.nz, d.L, leaves2, rho2)
    own_old = M.leaf_owner_map(d.nx, d.ny, d.nz, d.L, m.leaves)
    old_lvl = m.leaves[own_old[leaves2[:, 0], leaves2[:, 1], leaves2[:, 2]], 3]
    merged = (leaves2[:, 3] < old_lvl).astype(np.float64)
    assert merged.sum() == (fin == -1).sum() / 8
    same = A.rasterize(d.nx, d.ny, d.nz, d.L, leaves2, merged) == 0
    np.testing.assert_array_equal(new[same], old[same])


def test_adapt_rejects_bad_marks():
    dom = W.Domain(2, 1, 1, 1, 1.0)
    leaves = _children((0, 0, 0), 0, 1) + [[2, 0, 0, 0]]
    m = _mesh(dom, leaves)
    rho = np.full(m.Ne, 0.5)
    bad = np.zeros(m.Ne, np.int8)
    bad[0] = -1                                    # one sibling of eight
    with pytest.raises(ValueError):
        A.adapt(m, bad, rho)


# ---------------------------------------------------------------- Eq. 10
def test_design_difference_closed_forms():
    w = W.config1b(2)
    d = w.dom
    args = (d.nx, d.ny, d.nz, d.L)
    assert A.design_difference(*args, w.leaves, w.rho, w.leaves, w.rho) == 0.0
    assert A.design_difference(*args, w.leaves, w.rho, w.leaves, 2 * w.rho) == pytest.approx(1.0, rel=1e-14)
    assert A.design_difference(*args, w.leaves, w.rho, w.leaves, 0 * w.rho) == pytest.approx(1.0, rel=1e-14)
    # constant designs on different meshes: |a - b| / a
    u = W.uniform_leaves(d)
    assert A.design_difference(*args, w.leaves, np.full(len(w.leaves), 0.4), u,
                               np.full(len(u), 0.1)) == pytest.approx(0.75, rel=1e-14)
    # a refined copy (children inherit) is the same design
    m0 = _mesh(d, w.leaves)
    rho0 = w.rho[m0.perm]
    fin = np.where(m0.leaves[:, 3] < d.L, 1, 0).astype(np.int8)
    l2, r2 = A.adapt(m0, fin, rho0)
    assert l2.shape[0] == int(np.sum(np.where(m0.leaves[:, 3] < d.L, 8, 1)))
    assert A.design_difference(*args, m0.leaves, rho0, l2, r2) == 0.0


def test_design_difference_weights_by_volume():
    """One coarse leaf against its 8 children with different values: the integral weights
    each child by 1/8 of the parent's volume."""
    dom = W.Domain(1, 1, 1, 1, 1.0)
    coarse = np.array([[0, 0, 0, 0]])
    kids = np.array(_children((0, 0, 0), 0, 1))
    vals = np.arange(1.0, 9.0)
    dd = A.design_difference(1, 1, 1, 1, coarse, [4.5], kids, vals)
    assert dd == pytest.approx(np.abs(vals - 4.5).mean() / 4.5, rel=1e-15)


# ---------------------------------------------------------------- displacement transfer
def test_transfer_reproduces_linear_fields_and_is_the_identity_on_the_same_mesh():
    from oracle import fem as F
    w = W.config1b(2)
    d = w.dom
    m = _mesh(d, w.leaves)
    B = np.array([[0.5, -0.25, 1.0], [2.0, 0.75, -1.5], [-0.125, 0.3, 0.6]])
    a = np.array([0.3, -1.2, 2.0])
    lin = lambda p: a + p.astype(np.float64) @ B.T
    u_old = lin(m.nodes).ravel()
    # adapted mesh: refine everything below the finest level
    fin = np.where(m.leaves[:, 3] < d.L, 1, 0).astype(np.int8)
    l2, _ = A.adapt(m, fin, np.ones(m.Ne))
    m2 = _mesh(d, l2)
    got = A.transfer_field(m, u_old, m2.nodes)
    np.testing.assert_allclose(got, lin(m2.nodes), rtol=1e-13, atol=1e-13 * np.abs(lin(m2.nodes)).max())
    # same mesh: the nodal values come back
    rng = np.random.default_rng(1)
    uf = F.constraint_matrix(m) @ rng.standard_normal(F.constraint_matrix(m).shape[1])   # a C u field
    np.testing.assert_allclose(A.transfer_field(m, uf, m.nodes), uf.reshape(-1, 3), rtol=0, atol=1e-14)


def test_transfer_of_a_constrained_field_is_continuous_across_leaves():
    """A point on a face shared by leaves of different levels gets the same value from each."""
    from oracle import fem as F
    w = W.config1b(3)
    d = w.dom
    m = _mesh(d, w.leaves)
    C = F.constraint_matrix(m)
    uf = C @ np.random.default_rng(2).standard_normal(C.shape[1])
    # evaluate at every node through each leaf that contains it (closed box) and compare
    u = uf.reshape(-1, 3)
    for e in range(0, m.Ne, 7):
        lf = m.leaves[e]
        s = 1 << (d.L - int(lf[3]))
        for k in range(8):
            p = lf[:3] + s * np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1])
            got = A.transfer_field(m, uf, p[None])[0]
            np.testing.assert_allclose(got, u[m.conn[e, k]], rtol=1e-13, atol=1e-13 * np.abs(u).max())
