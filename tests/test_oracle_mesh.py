"""Pins for the oracle's mesh tables (paper Sec. 4, Sec. 6 Eq. 6, Fig. 3)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import fem as F
from oracle import mesh as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh(w, **kw):
    d = w.dom
    return M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces, **kw)


def test_morton_key_small_values():
    # bit i of x, y, z at 3i, 3i+1, 3i+2
    assert int(M.morton_key(1, 0, 0)) == 1
    assert int(M.morton_key(0, 1, 0)) == 2
    assert int(M.morton_key(0, 0, 1)) == 4
    assert int(M.morton_key(2, 0, 0)) == 8
    assert int(M.morton_key(3, 3, 3)) == 63
    assert int(M.morton_key(5, 0, 6)) == 0b101_100_001   # per bit level: (z y x)


def test_uniform_mesh_counts_and_no_hanging():
    dom = W.Domain(3, 2, 2, 0, 1.0)
    leaves = W.uniform_leaves(dom)
    m = M.build_mesh(3, 2, 2, 0, 1.0, leaves)
    assert m.Ne == 12
    assert m.Nn == 4 * 3 * 3
    assert len(m.hanging) == 0
    # every element's corner k sits at anchor + s*(i, j, m)
    for e in range(m.Ne):
        for k in range(8):
            assert tuple(m.nodes[m.conn[e, k]]) == tuple(m.leaves[e, :3] + M.CORNER_OFFSETS[k])
    # Dirichlet face x = 0 holds (ny+1)(nz+1) nodes
    assert m.dirichlet.sum() == 9


def _read_golden_hanging(path):
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = [p.split() for p in line.split("|")]
        h = tuple(int(v) for v in parts[0])
        out[h] = sorted((tuple(int(v) for v in p[:3]), Fraction(p[3])) for p in parts[1:])
    return out


def test_hanging_table_hand_derived():
    dom = W.Domain(2, 1, 1, 1, 1.0)
    leaves = W.refine(dom, W.uniform_leaves(dom), np.array([True, False]))
    m = M.build_mesh(2, 1, 1, 1, 1.0, leaves, dirichlet_faces=0)
    got = {tuple(m.nodes[h]): sorted((tuple(m.nodes[j]), w) for j, w in v) for h, v in m.hanging.items()}
    assert got == _read_golden_hanging(os.path.join(GOLDEN, "hanging_2x1x1_L1.txt"))
    assert m.Nn == 27 + 4


@pytest.mark.parametrize("make", [W.config1, W.config1b])
def test_hanging_matches_bruteforce(make):
    w = make()
    m = _mesh(w)
    bf = M.hanging_bruteforce(w.dom.nx, w.dom.ny, w.dom.nz, w.dom.L, w.leaves)
    got = {tuple(m.nodes[h]): sorted((tuple(m.nodes[j]), wt) for j, wt in v) for h, v in m.hanging.items()}
    assert got == bf
    assert len(got) > 0


@pytest.mark.parametrize("make", [W.config1, W.config1b, W.small_truss])
def test_mesh_invariants(make):
    w = make()
    m = _mesh(w)
    d = w.dom
    # volumes add up to the box
    assert np.isclose(m.volume.sum(), d.nx * d.ny * d.nz * d.h0 ** 3, rtol=1e-14)
    # canonical orders are Morton-sorted and unique
    ek = M.morton_key(m.leaves[:, 0], m.leaves[:, 1], m.leaves[:, 2])
    nk = M.morton_key(m.nodes[:, 0], m.nodes[:, 1], m.nodes[:, 2])
    assert (np.diff(ek.astype(np.float64)) > 0).all()
    assert (np.diff(nk.astype(np.float64)) > 0).all()
    # every node is used by some element
    assert np.bincount(m.conn.ravel(), minlength=m.Nn).min() >= 1
    # masters are never hanging on a balanced mesh; weights sum to one; 2 or 4 masters
    for h, ms in m.hanging.items():
        assert sum(wt for _, wt in ms) == 1
        assert len(ms) in (2, 4)
        for j, wt in ms:
            assert j not in m.hanging
            assert wt in (Fraction(1, 2), Fraction(1, 4))
    # the permutation maps input leaves to canonical order
    assert (w.leaves[m.perm] == m.leaves).all()


def test_rejects_invalid_leaf_sets():
    dom = W.Domain(2, 1, 1, 2, 1.0)
    ok = W.uniform_leaves(dom)
    M.check_leaves(2, 1, 1, 2, ok)
    with pytest.raises(ValueError):                      # gap
        M.check_leaves(2, 1, 1, 2, ok[:1])
    with pytest.raises(ValueError):                      # overlap
        M.check_leaves(2, 1, 1, 2, np.concatenate([ok, W.refine(dom, ok[:1], [True])[:1]]))
    with pytest.raises(ValueError):                      # misaligned anchor
        bad = ok.copy()
        bad[1, 0] += 1
        M.check_leaves(2, 1, 1, 2, bad)
    with pytest.raises(ValueError):                      # outside the box
        bad = ok.copy()
        bad[1, 1] = 4
        M.check_leaves(2, 1, 1, 2, bad)
    # level 2 next to level 0: not 2:1 balanced
    one = W.refine(dom, ok, [True, False])
    unbalanced = W.refine(dom, one, (one[:, 3] == 1) & (one[:, 0] == 2) & (one[:, 1] == 0) & (one[:, 2] == 0))
    M.check_leaves(2, 1, 1, 2, unbalanced)
    with pytest.raises(ValueError):
        M.check_balance(2, 1, 1, 2, unbalanced)
    W.balance(dom, unbalanced)   # the generator can repair it


def test_unbalanced_chains_resolve_to_linear_interpolation():
    # A level-2 leaf against a level-0 leaf: masters of hanging nodes can themselves hang.
    dom = W.Domain(2, 1, 1, 2, 1.0)
    one = W.refine(dom, W.uniform_leaves(dom), [True, False])
    sel = (one[:, 3] == 1) & (one[:, 0] == 2)
    leaves = W.refine(dom, one, sel)
    m = M.build_mesh(2, 1, 1, 2, 1.0, leaves, dirichlet_faces=0, validate=False)
    # a linear field is reproduced exactly at every hanging node by its resolved masters
    a = np.array([0.3, -1.7, 2.9])
    for h, ms in m.hanging.items():
        val = sum(float(wt) * (m.nodes[j] @ a) for j, wt in ms)
        assert abs(val - m.nodes[h] @ a) < 1e-12
        for j, _ in ms:
            assert j not in m.hanging


def test_trilinear_field_is_consistent_with_constraints():
    """Edge (linear) and face (bilinear) interpolation reproduce any trilinear field exactly; the
    field u = x (a + B (y, z)) vanishes on the clamped face, so Dirichlet masters agree too."""
    w = W.config1b()
    m = _mesh(w)
    X = m.nodes.astype(np.float64)
    a = np.array([0.1, -0.2, 0.3])
    B = np.array([[0.05, -0.2], [0.3, 0.1], [0.0, 0.25]])
    u = X[:, :1] * (a[None, :] + X[:, 1:] @ B.T)
    C = F.constraint_matrix(m)
    fn = F.free_nodes(m)
    uf = (C @ u[fn].ravel()).reshape(-1, 3)
    assert np.abs(uf - u).max() < 1e-12 * np.abs(u).max()
