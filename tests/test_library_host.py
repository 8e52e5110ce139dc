"""Host-side checks of libtm (no GPU): the library loads, exports every entry point
include/tm.h declares, and its integer mesh tables match the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import mesh as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tm():
    from paper_1009_4975_gb300 import build
    build.build()
    import paper_1009_4975_gb300 as P
    P.load_library()
    return P


def _declared():
    text = open(os.path.join(ROOT, "include", "tm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[A-Za-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(tm):
    lib = tm.load_library()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(tm.EXPORTS) == names


def _oracle_tables(w):
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    hn = m.hanging_ids()
    hm = np.full((hn.size, 4), -1, np.int64)
    for i, h in enumerate(hn):
        ms = [j for j, _ in m.hanging[h]]
        hm[i, :len(ms)] = ms
    flags = m.dirichlet.astype(np.uint8)
    flags[hn] |= 2
    return m, hn, hm, flags


@pytest.mark.parametrize("make", [W.config1, W.config1b, W.small_truss])
def test_tables_bit_exact_against_oracle(tm, make):
    w = make()
    d = w.dom
    info, t = tm.tm_tables_build(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    m, hn, hm, flags = _oracle_tables(w)
    assert info["Ne"] == m.Ne and info["Nn"] == m.Nn and info["n_hanging"] == hn.size
    assert np.array_equal(t["perm"], m.perm)
    assert np.array_equal(t["node_xyz"], m.nodes)
    assert np.array_equal(t["conn"], m.conn)
    assert np.array_equal(t["hang_node"], hn)
    assert np.array_equal(t["hang_master"], hm)
    assert np.array_equal(t["node_flags"], flags)
    fn = (flags == 0).sum()
    assert info["n_free"] == 3 * fn
    assert 0 < info["max_local"] <= 1024


def _morton(x, y, z):
    k = 0
    for b in range(21):
        k |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    return k


def test_tables_bit_exact_on_a_sparse_key_space(tm):
    """A long thin domain (1 x 1 x 160 base cells, two levels of refinement with hanging nodes):
    its corner Morton keys span far more 64-bit words than 8 per element, so the library numbers
    the nodes by sorting the keys instead of ranking them in a bitmap of the key space.  Both give
    the sorted distinct keys; the tables still equal the oracle's."""
    dom = W.Domain(1, 1, 160, 2, 1.0)
    rng = np.random.default_rng(5)
    lv = W.uniform_leaves(dom)
    lv = W.refine(dom, lv, rng.random(len(lv)) < 0.3)
    lv = W.balance(dom, W.refine(dom, lv, (lv[:, 3] == 1) & (rng.random(len(lv)) < 0.3)))
    fx, fy, fz = dom.fine_shape
    assert _morton(fx, fy, fz) // 64 + 1 > max(1 << 16, 8 * len(lv))
    info, t = tm.tm_tables_build(dom.nx, dom.ny, dom.nz, dom.L, dom.h0, lv)
    m = M.build_mesh(dom.nx, dom.ny, dom.nz, dom.L, dom.h0, lv)
    hn = m.hanging_ids()
    assert info["Nn"] == m.Nn and info["n_hanging"] == hn.size > 0
    assert np.array_equal(t["node_xyz"], m.nodes)
    assert np.array_equal(t["conn"], m.conn)
    assert np.array_equal(t["hang_node"], hn)


def test_tables_other_dirichlet_faces(tm):
    w = W.config1()
    d = w.dom
    faces = 0b100101          # x = 0, y = 0, z = max
    info, t = tm.tm_tables_build(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=faces)
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=faces)
    assert np.array_equal(t["node_flags"] & 1, m.dirichlet.astype(np.uint8))


def test_rejects_invalid_leaf_sets(tm):
    dom = W.Domain(2, 1, 1, 2, 1.0)
    ok = W.uniform_leaves(dom)
    tm.tm_tables_build(2, 1, 1, 2, 1.0, ok)
    cases = {
        "gap": ok[:1],
        "overlap": np.concatenate([ok, W.refine(dom, ok[:1], [True])[:1]]),
        "misaligned": ok + np.array([[0, 0, 0, 0], [1, 0, 0, 0]]),
        "outside": ok + np.array([[0, 0, 0, 0], [0, 4, 0, 0]]),
        "level": ok + np.array([[0, 0, 0, 3], [0, 0, 0, 0]]),
    }
    one = W.refine(dom, ok, [True, False])
    cases["unbalanced"] = W.refine(dom, one, (one[:, 3] == 1) & (one[:, 0] == 2) & (one[:, 1] == 0) & (one[:, 2] == 0))
    for name, lv in cases.items():
        with pytest.raises(tm.TmError) as ei:
            tm.tm_tables_build(2, 1, 1, 2, 1.0, lv)
        assert ei.value.code == tm.TM_EINVAL, name
    # the balanced repair is accepted
    tm.tm_tables_build(2, 1, 1, 2, 1.0, W.balance(dom, cases["unbalanced"]))


def test_python_binding_fails_loudly_without_gpu(tm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tm.TmError):
        tm.tm_create(0, stream=0)


def test_tables_do_not_depend_on_the_number_of_host_threads(tm, monkeypatch):
    """The table build and the adaptation's new leaf set split their passes over host threads
    (at most one per 65,536 items, limited by TM_HOST_THREADS) and merge the chunks in order.  On a
    202k-leaf truss mesh (bricks, blocks, hanging nodes) every exported table and the adapted leaf
    set are the same bytes with 1, 3 and the default number of threads."""
    w = W.small_truss(seed=3, base=(32, 16, 16), L=2)
    d = w.dom
    rng = np.random.default_rng(8)
    mark = ((w.leaves[:, 3] < d.L) & (rng.random(len(w.leaves)) < 0.05)).astype(np.int8)
    rho = rng.uniform(1e-3, 1.0, len(w.leaves))

    def everything(nthreads):
        if nthreads is None:
            monkeypatch.delenv("TM_HOST_THREADS", raising=False)
        else:
            monkeypatch.setenv("TM_HOST_THREADS", str(nthreads))
        info, t = tm.tm_tables_build(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
        ops = tm.tm_tables_operator(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces)
        # the adaptation takes the leaves in canonical (Morton) order
        leaves = np.asarray(w.leaves)[t["perm"]]
        al, ar = tm.tm_tables_adapt(d.nx, d.ny, d.nz, d.L, d.h0, leaves, mark[t["perm"]], rho[t["perm"]])
        arrays = dict(t)
        arrays.update({k: v for k, v in ops.items() if isinstance(v, np.ndarray)})
        arrays.update(adapt_leaves=np.asarray(al), adapt_rho=np.asarray(ar))
        return info, ops["info"], arrays

    ref_info, ref_ops_info, ref = everything(1)
    assert ref_info["Ne"] > 3 * 65536 and ref_info["n_blocks"] > 100 and ref_info["n_bricks"] > 1000
    assert ref_info["n_hanging"] > 0
    for n in (3, None):
        info, ops_info, got = everything(n)
        assert info == ref_info and ops_info == ref_ops_info
        assert got.keys() == ref.keys()
        for k in ref:
            assert got[k].dtype == ref[k].dtype and got[k].tobytes() == ref[k].tobytes(), (n, k)


@pytest.mark.parametrize("make", [W.config1b, W.small_truss])
def test_jacobi_diagonal_tables_against_the_assembled_matrix(tm, make):
    """The Jacobi diagonal the library's tables give (sum over a node's entries of c_e times a
    tabulated triple v^T K0 v, Sec. 5) equals the diagonal of the oracle's assembled C^T K C at
    every free DOF, for random densities, on meshes with edge- and face-hanging nodes."""
    from oracle import fem as F
    w = make()
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    rng = np.random.default_rng(11)
    rho = rng.uniform(1e-3, 1.0, m.Ne)
    A, _, _ = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val, w.E0, w.Emin, w.nu, w.penal)
    g = tm.tm_tables_diag(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, nu=w.nu)
    assert g["info"]["n_hanging"] > 0
    ptr, elem, q, tab = g["ptr"], g["elem"], g["q"], g["tab"]
    assert ptr[0] == 0 and np.all(np.diff(ptr) >= 0) and ptr[-1] == elem.size == q.size
    assert int(q.max()) < tab.shape[0]
    ce = (w.Emin + rho ** w.penal * (w.E0 - w.Emin)) * (d.h0 / 2.0 ** m.leaves[:, 3])
    node = np.repeat(np.arange(m.Nn), np.diff(ptr))
    dfull = np.zeros((m.Nn, 3))
    np.add.at(dfull, node, ce[elem][:, None] * tab[q])
    got = F.from_full_layout(m, dfull.ravel())
    np.testing.assert_allclose(got, A.diagonal(), rtol=1e-13, atol=0)
    # ascending elements within every node, and every element-node incidence listed once
    same = node[1:] == node[:-1]
    assert np.all(elem[1:][same] > elem[:-1][same])


_NOMEM_CHILD = r"""
import resource, sys
import numpy as np
import paper_1009_4975_gb300 as P
P.load_library()
nx, ny, nz = 128, 128, 64
g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
leaves = np.ascontiguousarray(np.concatenate([g, np.zeros((len(g), 1), np.int64)], 1).astype(np.int32))
vm = [int(l.split()[1]) * 1024 for l in open("/proc/self/status") if l.startswith("VmSize")][0]
cap = vm + (int(sys.argv[1]) << 20)
resource.setrlimit(resource.RLIMIT_AS, (cap, cap))
try:
    info, _ = P.tm_tables_build(nx, ny, nz, 0, 1.0, leaves)
    print("built", info["Ne"])
except P.TmError as e:
    print("status", e.code, str(e))
"""


@pytest.mark.parametrize("headroom_mb", [16, 200, 500, 4000])
def test_host_allocation_failure_is_a_status_not_an_abort(headroom_mb):
    """A C++ exception must not cross the C ABI.  A child process whose address space is capped a
    little above its size at the call builds the tables of a 1M-leaf mesh: where the cap cuts the
    build off (in the calling thread, in a worker thread or at a thread's start), tm_tables_build
    returns TM_ENOMEM with a message and the process lives on; with room enough it builds."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _NOMEM_CHILD, str(headroom_mb)], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout.split()
    if headroom_mb >= 4000:
        assert out[:2] == ["built", str(128 * 128 * 64)]
    else:
        import paper_1009_4975_gb300 as P
        assert out[:2] == ["status", str(P.TM_ENOMEM)], r.stdout
        assert "host memory allocation failed" in r.stdout
