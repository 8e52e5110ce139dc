"""Host form of the adaptation step (tm_tables_adapt, no GPU) against the oracle: the new
leaves and densities must match bit for bit, and malformed marks must be rejected."""
import numpy as np
import pytest

import workloads as W
from oracle import amr as A
from oracle import mesh as M


@pytest.fixture(scope="module")
def tm():
    from paper_1009_4975_gb300 import build
    build.build()
    import paper_1009_4975_gb300 as P
    P.load_library()
    return P


def _case(seed):
    w = W.config1b(seed)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    phi = W.truss_sdf(m.centres, seed + 7, r0=0.09)
    rho = np.clip(0.5 - phi / (2.0 * d.h_min), 1e-3, 1.0)
    return w, m, rho


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_adapt_matches_oracle_bit_exact(tm, seed):
    w, m, rho = _case(seed)
    d = w.dom
    marks = A.final_marks(m, rho, 0.5, 1.6 * d.h_min)
    want_l, want_r = A.adapt(m, marks, rho)
    got_l, got_r = tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, marks, rho)
    np.testing.assert_array_equal(got_l, want_l)
    assert got_r.tobytes() == want_r.tobytes()


def test_adapt_refine_everything_and_nothing(tm):
    w, m, rho = _case(1)
    d = w.dom
    keep = np.zeros(m.Ne, np.int8)
    gl, gr = tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, keep, rho)
    np.testing.assert_array_equal(gl, m.leaves)
    assert gr.tobytes() == rho.tobytes()
    up = np.where(m.leaves[:, 3] < d.L, 1, 0).astype(np.int8)
    gl, gr = tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, up, rho)
    wl, wr = A.adapt(m, up, rho)
    np.testing.assert_array_equal(gl, wl)
    assert gr.tobytes() == wr.tobytes()


def test_adapt_rejects_malformed_marks(tm):
    w, m, rho = _case(2)
    d = w.dom
    fin = m.leaves[:, 3] == d.L
    bad = np.zeros(m.Ne, np.int8)
    bad[np.nonzero(fin)[0][0]] = 1                      # refine past the finest level
    with pytest.raises(tm.TmError):
        tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, bad, rho)
    bad = np.zeros(m.Ne, np.int8)
    bad[np.nonzero(m.leaves[:, 3] > 0)[0][3]] = -1      # one sibling of a family
    with pytest.raises(tm.TmError):
        tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, bad, rho)
    u = W.uniform_leaves(d)
    mu = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, u)
    bad = -np.ones(mu.Ne, np.int8)                      # level 0 cannot derefine
    with pytest.raises(tm.TmError):
        tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, mu.leaves, bad, np.full(mu.Ne, 0.5))


def test_transfer_matches_the_oracle(tm):
    """The library's host transfer of a constrained field to the nodes of an adapted mesh
    equals the oracle's evaluation (same trilinear sums, to rounding)."""
    from oracle import fem as F
    w, m, rho = _case(1)
    d = w.dom
    C = F.constraint_matrix(m)
    uf = C @ np.random.default_rng(6).standard_normal(C.shape[1])
    marks = A.final_marks(m, rho, 0.5, 1.6 * d.h_min)
    l2, _ = A.adapt(m, marks, rho)
    m2 = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, l2)
    want = A.transfer_field(m, uf, m2.nodes)
    got = tm.tm_tables_transfer(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, uf, m2.nodes)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-14 * np.abs(uf).max())
    with pytest.raises(tm.TmError):
        tm.tm_tables_transfer(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, uf, [[-1, 0, 0]])


def test_adapt_on_several_host_threads(tm):
    """A mesh of over 65,536 leaves, which the library splits into element chunks on several host
    threads: refinement, derefinement and the 2:1 balancing still equal the oracle bit for bit,
    and a malformed mark in the last chunk alone is still rejected."""
    w = W.small_truss(seed=2, base=(24, 12, 12), L=2)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    assert m.Ne > 65536
    phi = W.truss_sdf(m.centres, 9, r0=0.09)
    rho = np.clip(0.5 - phi / (2.0 * d.h_min), 1e-3, 1.0)
    marks = A.final_marks(m, rho, 0.5, 1.6 * d.h_min)
    rng = np.random.default_rng(3)
    marks = np.where((marks == 0) & (m.leaves[:, 3] < d.L) & (rng.random(m.Ne) < 0.02), 1, marks).astype(np.int8)
    assert (marks == 1).sum() > 100 and (marks == -1).sum() > 1000
    want_l, want_r = A.adapt(m, marks, rho)
    got_l, got_r = tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, marks, rho)
    np.testing.assert_array_equal(got_l, want_l)
    assert got_r.tobytes() == want_r.tobytes()
    bad = marks.copy()
    e = np.nonzero(m.leaves[:, 3] == d.L)[0][-1]         # refine past the finest level, near the end
    bad[e] = 1
    with pytest.raises(tm.TmError):
        tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, m.leaves, bad, rho)
