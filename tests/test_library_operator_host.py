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
    hdr = rec[:64].view(np.int32)
    (e0, ne, nreg, nsh, nhang, ninv, o_lslot, o_hent, o_iptr, o_inv, o_lcorner, o_lnode, o_elist,
     *pad) = (int(v) for v in hdr)
    assert pad == [0, 0, 0]
    nloc = nreg + nhang
    return dict(
        e0=e0, ne=ne, nreg=nreg, nsh=nsh, nhang=nhang,
        elist=rec[o_elist:o_elist + 4 * ne].view(np.int32).astype(np.int64),
        lcorner=rec[o_lcorner:o_lcorner + 16 * ne].view(np.uint16).reshape(ne, 8).astype(np.int64),
        lnode=rec[o_lnode:o_lnode + 4 * nreg].view(np.uint32).astype(np.int64),
        lslot=rec[o_lslot:o_lslot + 4 * nsh].view(np.int32).astype(np.int64),
        hent=rec[o_hent:o_hent + 8 * nhang].view(np.uint16).reshape(nhang, 4).astype(np.int64),
        iptr=rec[o_iptr:o_iptr + 2 * (nloc + 1)].view(np.uint16).astype(np.int64),
        inv=rec[o_inv:o_inv + 2 * ninv].view(np.uint16).astype(np.int64),
        offsets=(o_lslot, o_hent, o_iptr, o_inv, o_lcorner, o_lnode, o_elist))


def _demorton(t):
    return (t & 1) | ((t >> 2) & 2), ((t >> 1) & 1) | ((t >> 3) & 2), ((t >> 2) & 1) | ((t >> 4) & 2)


def _lat(a, b, c):
    return a + 5 * b + 25 * c


def _brick_masters(nd, mask):
    """Lattice nodes one step away from hanging lattice node nd along the axes in mask."""
    p = np.array([nd % 5, (nd // 5) % 5, nd // 25])
    axes = [a for a in range(3) if mask >> a & 1]
    out = []
    for signs in np.ndindex(*([2] * len(axes))):
        q = p.copy()
        for a, sg in zip(axes, signs):
            q[a] += 1 if sg else -1
        out.append(_lat(*q))
    return out


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
        Y = ce[B["elist"], None] * _modal_product(ops["modal"], X)
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
    for bi in range(len(ops["brick_e0"])):                      # bricks: the 5x5x5 lattice
        e0, node, hax, out = (ops["brick_e0"][bi], ops["brick_node"][bi].astype(np.int64) & 0xFFFFFFFF,
                              ops["brick_hax"][bi], ops["brick_out"][bi])
        g = node & 0x7FFFFFFF
        fixed = (node >> 31).astype(bool)
        R = np.where(fixed[:, None], 0.0, x[g])
        for nd in np.nonzero(hax)[0]:                            # C: masters one step away
            ms = _brick_masters(nd, hax[nd])
            R[nd] = sum(R[q] for q in ms) / len(ms)
        S = np.zeros((125, 3))
        for t in range(64):
            i, j, k = _demorton(t)
            corners = [_lat(i + (q & 1), j + ((q >> 1) & 1), k + (q >> 2)) for q in range(8)]
            Y = ce[e0 + t] * _modal_product(ops["modal"], R[corners].reshape(1, 24))[0]
            for q, nd in enumerate(corners):
                S[nd] += Y[3 * q:3 * q + 3]
        for nd in np.nonzero(hax)[0]:                            # C^T: fold into the masters
            ms = _brick_masters(nd, hax[nd])
            for q in ms:
                S[q] += S[nd] / len(ms)
        for nd in range(125):
            if hax[nd]:
                assert out[nd] == -2
                continue
            s = np.zeros(3) if fixed[nd] else S[nd]
            if out[nd] >= 0:
                part[out[nd]] = s
            else:
                assert out[nd] == -1
                y[g[nd]] = s
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
    assert ro[0] == 0 and np.all(np.diff(ro) > 0)
    hang = set(int(h) for h in m.hanging_ids())
    owners = np.zeros(m.Nn, np.int64)            # blocks and bricks that hold each regular node
    covered = np.zeros(m.Ne, np.int64)
    e_last = -1
    for b in range(len(ro) - 1):
        B = _parse(ops["brec"], ro[b], ro[b + 1])
        el = B["elist"]                                      # ascending over all blocks
        assert 1 <= B["ne"] <= 256 and el[0] == B["e0"] and el[0] > e_last and np.all(np.diff(el) > 0)
        e_last = el[-1]
        covered[el] += 1
        o_lslot, o_hent, o_iptr, o_inv, o_lcorner, o_lnode, o_elist = B["offsets"]
        assert o_lcorner == 64 and o_elist == 64 + 16 * B["ne"]
        assert o_lnode % 4 == 0 and o_lslot % 4 == 0 and o_hent % 8 == 0
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
        conn = m.conn[B["elist"]]
        for t in range(B["ne"]):
            for k in range(8):
                loc = B["lcorner"][t, k]
                if loc < B["nreg"]:
                    assert g[loc] == conn[t, k]
                else:
                    assert int(conn[t, k]) in hang
    # bricks: aligned 4x4x4 cubes of one level, 64 consecutive elements in Morton order, whose
    # lattice names the elements' corners; hanging lattice nodes interpolate lattice neighbours
    assert ops["info"]["n_bricks"] == len(ops["brick_e0"])
    slots = []
    for bi, e0 in enumerate(ops["brick_e0"]):
        covered[e0:e0 + 64] += 1
        lv = m.leaves[e0:e0 + 64]
        s = 1 << (m.L - int(lv[0, 3]))
        assert np.all(lv[:, 3] == lv[0, 3]) and np.all(lv[0, :3] % (4 * s) == 0)
        node = ops["brick_node"][bi].astype(np.int64) & 0x7FFFFFFF
        hax, out = ops["brick_hax"][bi], ops["brick_out"][bi]
        for t in range(64):
            ijk = np.array(_demorton(t))
            assert np.array_equal(lv[t, :3], lv[0, :3] + s * ijk)
            for q in range(8):
                nd = _lat(ijk[0] + (q & 1), ijk[1] + ((q >> 1) & 1), ijk[2] + (q >> 2))
                assert node[nd] == m.conn[e0 + t, q]
        for nd in range(125):
            n = int(node[nd])
            assert bool(ops["brick_node"][bi][nd] < 0) == bool(m.dirichlet[n])
            if n in hang:
                assert hax[nd] != 0 and out[nd] == -2
                ms = sorted(int(node[q]) for q in _brick_masters(nd, hax[nd]))
                assert ms == sorted(int(mm) for mm, _ in m.hanging[n])
                assert ops["brick_fold"][bi][nd] == 0
            else:
                assert hax[nd] == 0 and out[nd] >= -1
                owners[n] += 1
                # fold mask: exactly the hanging lattice nodes this node is a master of
                want = set(h for h in range(125) if hax[h] and nd in _brick_masters(h, hax[h]))
                got = set()
                fm = int(ops["brick_fold"][bi][nd])
                a, b, c = nd % 5, (nd // 5) % 5, nd // 25
                for bit in range(18):
                    if not fm >> bit & 1:
                        continue
                    if bit < 6:
                        d = [0, 0, 0]
                        d[bit >> 1] = 1 if bit & 1 else -1
                    else:
                        pl, bb = (bit - 6) >> 2, bit - 6
                        ax0, ax1 = (0, 1) if pl == 0 else ((0, 2) if pl == 1 else (1, 2))
                        d = [0, 0, 0]
                        d[ax0] = 1 if bb & 1 else -1
                        d[ax1] = 1 if bb & 2 else -1
                    got.add(_lat(a + d[0], b + d[1], c + d[2]))
                assert got == want, (bi, nd, got, want)
                if out[nd] >= 0:
                    slots.append(int(out[nd]))
    assert np.all(covered == 1)                  # blocks and bricks partition the elements
    # shared nodes (in more than one block or brick) have one partial per holder, node-major
    sh = ops["sh_node"]
    assert np.array_equal(np.sort(sh), np.nonzero(owners > 1)[0])
    assert np.array_equal(np.diff(ops["sh_ptr"]), owners[sh])
    # brick partial slots are distinct and within the shared-node ranges
    assert len(set(slots)) == len(slots) and (not slots or max(slots) < ops["sh_ptr"][-1])
    for bi in range(len(ops["brick_e0"])):
        node = ops["brick_node"][bi].astype(np.int64) & 0x7FFFFFFF
        for nd in range(125):
            o = int(ops["brick_out"][bi][nd])
            if o >= 0:
                i = int(np.searchsorted(sh, node[nd]))
                assert sh[i] == node[nd] and ops["sh_ptr"][i] <= o < ops["sh_ptr"][i + 1]
            elif o == -1:
                assert owners[node[nd]] == 1
