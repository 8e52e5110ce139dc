"""Host-side check of the operator's block tables (no GPU): the records the library builds for
its operator kernel are interpreted here step by step, as the kernel uses them:
- hanging values interpolated from their masters;
- element products c_e K0 X_e via the exported symmetry-adapted blocks;
- per-node slot sums and folds of hanging sums into masters;
- partials of block-shared nodes summed node-major.

The result must equal the oracle's assembled A x = C^T K C x.  The exported modal blocks must
reproduce the oracle's K0, and the tables must satisfy their structural invariants."""
import numpy as np
import pytest

import workloads as W
from oracle import fem as F
from oracle import mesh as M

U64 = np.finfo(np.float64).eps
SLOT_ROW = 25
FOLD, QUARTER = 0x8000, 0x4000


@pytest.fixture(scope="module")
def tm():
    from paper_1009_4975_gb300 import build
    build.build()
    import paper_1009_4975_gb300 as P
    P.load_library()
    return P


def _butterfly(v):
    """T x per component: along each axis (bit 1, 2, 4) (a, b) -> (a + b, b - a)."""
    v = v.copy()
    for bit in (1, 2, 4):
        for k in range(8):
            if not k & bit:
                a, b = v[..., k].copy(), v[..., k | bit].copy()
                v[..., k], v[..., k | bit] = a + b, b - a
    return v


def _butterfly_t(v):
    """T^T z: the transposed stages (s, d) -> (s - d, s + d), in reverse order."""
    v = v.copy()
    for bit in (1, 2, 4):
        for k in range(8):
            if not k & bit:
                s_, d_ = v[..., k].copy(), v[..., k | bit].copy()
                v[..., k], v[..., k | bit] = s_ - d_, s_ + d_
    return v


def _modal_product(modal, X):
    """K0 X for a batch X (n, 24) (DOF 3k + c) through the symmetry-adapted blocks."""
    w = _butterfly(X.reshape(-1, 8, 3).transpose(0, 2, 1))       # (n, 3, 8)
    z = np.zeros_like(w)
    for s in range(8):
        a = np.stack([w[:, 0, s ^ 1], w[:, 1, s ^ 2], w[:, 2, s ^ 4]], axis=1)    # (n, 3)
        r = a @ modal[s].T
        z[:, 0, s ^ 1], z[:, 1, s ^ 2], z[:, 2, s ^ 4] = r[:, 0], r[:, 1], r[:, 2]
    return _butterfly_t(z).transpose(0, 2, 1).reshape(-1, 24)


def test_modal_blocks_reproduce_the_oracle_element_matrix(tm):
    w = W.config1()
    d = w.dom
    modal = tm.tm_tables_operator(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)["modal"]
    K0 = F.reference_stiffness(0.3)
    got = _modal_product(modal, np.eye(24))
    assert np.abs(got - K0).max() <= 64 * U64 * np.abs(K0).max()
    # translation rows and columns vanish: blocks 1, 2, 4 act as 2 x 2
    for s, c in ((1, 0), (2, 1), (4, 2)):
        assert np.all(modal[s][c, :] == 0) and np.all(modal[s][:, c] == 0)


def _parse(brec, r0, r1):
    rec = brec[16 * r0:16 * r1]
    hdr = rec[:48].view(np.int32)
    e0, ne, nreg, nsh, nhang, ninv, o_lslot, o_hent, o_iptr, o_inv, o_lcorner, o_lnode = (int(v) for v in hdr)
    nloc = nreg + nhang
    return dict(
        e0=e0, ne=ne, nreg=nreg, nsh=nsh, nhang=nhang,
        lcorner=rec[o_lcorner:o_lcorner + 16 * ne].view(np.uint16).reshape(ne, 8).astype(np.int64),
        lnode=rec[o_lnode:o_lnode + 4 * nreg].view(np.uint32).astype(np.int64),
        lslot=rec[o_lslot:o_lslot + 4 * nsh].view(np.int32).astype(np.int64),
        hent=rec[o_hent:o_hent + 8 * nhang].view(np.uint16).reshape(nhang, 4).astype(np.int64),
        iptr=rec[o_iptr:o_iptr + 2 * (nloc + 1)].view(np.uint16).astype(np.int64),
        inv=rec[o_inv:o_inv + 2 * ninv].view(np.uint16).astype(np.int64),
        offsets=(o_lslot, o_hent, o_iptr, o_inv, o_lcorner, o_lnode))


def _interpret(ops, m, rho, x_full, E0=1.0, Emin=1e-9, penal=3.0):
    """y = C^T K C x from the exported tables, as the operator kernel computes it."""
    ce = F.young(rho, E0, Emin, penal) * m.h
    x = x_full.reshape(-1, 3)
    y = np.zeros_like(x)
    nsh_total = ops["sh_ptr"][-1]
    part = np.full((nsh_total, 3), np.nan)
    ro = ops["rec_off"]
    for b in range(len(ro) - 1):
        B = _parse(ops["brec"], ro[b], ro[b + 1])
        nreg, nhang = B["nreg"], B["nhang"]
        g = B["lnode"] & 0x7FFFFFFF
        fixed = (B["lnode"] >> 31).astype(bool)
        R = np.zeros((nreg + nhang, 3))
        R[:nreg] = np.where(fixed[:, None], 0.0, x[g])
        for j in range(nhang):                                   # C: interpolation
            ms = [int(v) for v in B["hent"][j] if v != 0xFFFF]
            R[nreg + j] = sum(R[q] for q in ms) / len(ms)
        X = R[B["lcorner"]].reshape(B["ne"], 24)                # element products
        Y = ce[B["e0"]:B["e0"] + B["ne"], None] * _modal_product(ops["modal"], X)
        XY = np.zeros((B["ne"] * SLOT_ROW + 3,))
        for t in range(B["ne"]):
            XY[t * SLOT_ROW:t * SLOT_ROW + 24] = Y[t]
        ip, iv = B["iptr"], B["inv"]
        H = np.zeros((nhang, 3))
        for j in range(nhang):                                   # hanging sums
            for p in iv[ip[nreg + j]:ip[nreg + j + 1]]:
                assert not p & FOLD
                H[j] += XY[p:p + 3]
        for i in range(nreg):                                    # C^T: slots and folds
            s = np.zeros(3)
            for p in iv[ip[i]:ip[i + 1]]:
                if p & FOLD:
                    s += (0.25 if p & QUARTER else 0.5) * H[p & (QUARTER - 1)]
                else:
                    s += XY[p:p + 3]
            if fixed[i]:
                s[:] = 0.0
            if i < B["nsh"]:
                part[B["lslot"][i]] = s
            else:
                y[g[i]] = s
    for i, n in enumerate(ops["sh_node"]):                       # second pass, node-major
        y[n] = part[ops["sh_ptr"][i]:ops["sh_ptr"][i + 1]].sum(axis=0)
    y[m.hanging_ids()] = 0.0
    return y.ravel()


CASES = {"config1": lambda: W.config1(), "config1b": lambda: W.config1b(),
         "truss_8x4x4_L2": lambda: W.small_truss(seed=4, base=(8, 4, 4), L=2)}


@pytest.mark.parametrize("name", list(CASES))
def test_block_tables_reproduce_the_assembled_operator(tm, name):
    w = CASES[name]()
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    ops = tm.tm_tables_operator(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces)
    rho = w.rho[m.perm]
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val)
    x = np.random.default_rng(5).standard_normal(A.shape[0])
    y = _interpret(ops, m, rho, F.to_full_layout(m, x))
    err = np.abs(F.from_full_layout(m, y) - A @ x)
    assert np.all(err <= 256 * U64 * (abs(A) @ np.abs(x)))


@pytest.mark.parametrize("name", list(CASES))
def test_block_table_invariants(tm, name):
    w = CASES[name]()
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    ops = tm.tm_tables_operator(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces)
    ro = ops["rec_off"]
    assert ops["info"]["n_blocks"] == (m.Ne + 255) // 256 and ro[0] == 0 and np.all(np.diff(ro) > 0)
    hang = set(int(h) for h in m.hanging_ids())
    owners = np.zeros(m.Nn, np.int64)            # blocks that hold each regular node
    e_next = 0
    for b in range(len(ro) - 1):
        B = _parse(ops["brec"], ro[b], ro[b + 1])
        assert B["e0"] == e_next and 1 <= B["ne"] <= 256
        e_next += B["ne"]
        o_lslot, o_hent, o_iptr, o_inv, o_lcorner, o_lnode = B["offsets"]
        assert o_lcorner == 48 and o_lnode % 4 == 0 and o_lslot % 4 == 0 and o_hent % 8 == 0
        assert o_iptr % 2 == 0 and o_inv % 2 == 0 and (ro[b + 1] - ro[b]) * 16 >= o_inv + 2 * len(B["inv"])
        g = B["lnode"] & 0x7FFFFFFF
        assert len(set(g.tolist())) == B["nreg"] and not (set(g.tolist()) & hang)
        owners[g] += 1
        # every (element, corner) slot appears exactly once, in the list of the local node
        # that corner maps to
        seen = {}
        ip, iv = B["iptr"], B["inv"]
        for i in range(B["nreg"] + B["nhang"]):
            for p in iv[ip[i]:ip[i + 1]]:
                if p & FOLD:
                    continue
                assert p < QUARTER and p % SLOT_ROW < 24 and (p % SLOT_ROW) % 3 == 0
                t, k = p // SLOT_ROW, (p % SLOT_ROW) // 3
                assert (t, k) not in seen and B["lcorner"][t, k] == i
                seen[(t, k)] = i
        assert len(seen) == 8 * B["ne"]
        # local corners name the element's global nodes
        conn = m.conn[B["e0"]:B["e0"] + B["ne"]]
        for t in range(B["ne"]):
            for k in range(8):
                loc = B["lcorner"][t, k]
                if loc < B["nreg"]:
                    assert g[loc] == conn[t, k]
                else:
                    assert int(conn[t, k]) in hang
    assert e_next == m.Ne
    # shared nodes (in more than one block) have one partial per block, node-major
    sh = ops["sh_node"]
    assert np.array_equal(np.sort(sh), np.nonzero(owners > 1)[0])
    assert np.array_equal(np.diff(ops["sh_ptr"]), owners[sh])
