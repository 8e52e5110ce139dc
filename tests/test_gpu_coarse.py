"""The two-level preconditioner on the GPU against the oracle (oracle/coarse.py), through the C ABI.

* Level operators: the GPU's cell matrices (built from moments of E over the cells), assembled
  on the host, equal the oracle's Galerkin products P0^T A P0 and P^T A_l P.  They are computed
  in FP64 and stored in FP32, so each assembled entry is within 4 u32 of the sum of the absolute
  cell entries that meet in it.
* Transfers and level products: FP32 sums of at most a few hundred terms, within 64 u32 of the
  sum of the absolute terms.
* One V-cycle: the GPU's FP32 cycle against the oracle's FP64 cycle, relative 2-norm error below
  1e-4 (FP32 rounding through the sweeps and the coarsest solve; the cycle is a preconditioner,
  and its effect on the solve is checked separately).
* Solves: the two-level mixed solve reaches a residual of 1e-8 in the oracle's A, in a fraction
  of the Jacobi iterations.
"""
import numpy as np
import pytest

from oracle import coarse as CO
from tests.gpu_common import U32, case, ctx, tm

pytestmark = pytest.mark.gpu


def _setup(name):
    c = case(name)
    c.upload()
    rho = c.t(c.rho)
    info = tm().tm_coarse_setup(ctx(), rho)
    H = CO.Hierarchy(c.m, c.A, c.w.dirichlet_faces)
    return c, rho, info, H


def _lattice_free(shape):
    return CO._dofs(CO.lattice_free(shape, 1))


def _embed(shape, v):
    X, Y, Z = shape
    out = np.zeros(3 * (X + 1) * (Y + 1) * (Z + 1))
    out[_lattice_free(shape)] = v
    return out


@pytest.mark.parametrize("name", ["config1b", "small_truss", "truss_10x5x5_L1"])
def test_level_operators_match_the_oracle_galerkin_products(name):
    import torch
    c, rho, info, H = _setup(name)
    assert info["levels"] == H.levels
    assert [tuple(s) for s in info["shapes"]] == [tuple(s) for s in H.shapes]
    for l, shape in enumerate(H.shapes):
        X, Y, Z = shape
        K = torch.zeros(X * Y * Z * 576, dtype=torch.float32, device="cuda")
        tm().tm_coarse_cells(ctx(), l, K)
        Kh = K.double().cpu().numpy().reshape(-1, 24, 24)
        A = CO.assemble_cells(shape, Kh)
        scale = CO.assemble_cells(shape, np.abs(Kh))
        diff = np.abs(A.toarray() - H.A[l].toarray())
        bound = 4 * U32 * scale.toarray()
        assert np.all(diff <= bound), (l, (diff - bound).max())
        assert np.allclose(Kh, Kh.transpose(0, 2, 1))


@pytest.mark.parametrize("name", ["config1b", "small_truss", "truss_10x5x5_L1"])
def test_restriction_prolongation_and_level_products_match_the_oracle(name):
    import torch
    c, rho, info, H = _setup(name)
    rng = np.random.default_rng(31)
    n = c.A.shape[0]
    r = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    rd = c.t(c.full(r), torch.float32)
    shape0 = H.shapes[0]
    n0 = 3 * np.prod(np.array(shape0) + 1)
    b0 = torch.zeros(n0, dtype=torch.float32, device="cuda")
    tm().tm_coarse_restrict(ctx(), rd, b0)
    got = b0.double().cpu().numpy()
    want = _embed(shape0, H.P0.T @ r)
    tol = 64 * U32 * _embed(shape0, abs(H.P0).T @ np.abs(r))
    assert np.all(np.abs(got - want) <= tol)
    # prolongation of a level-0 vector (zero at clamped lattice nodes)
    v = np.zeros(n0)
    v[_lattice_free(shape0)] = rng.standard_normal(_lattice_free(shape0).size).astype(np.float32)
    vd = c.t(v, torch.float32)
    y = torch.full((3 * c.m.Nn,), 9.0, dtype=torch.float32, device="cuda")
    tm().tm_coarse_prolong(ctx(), vd, y)
    gy = y.double().cpu().numpy()
    vf = v[_lattice_free(shape0)]
    wy = c.full(H.P0 @ vf)
    ty = 16 * U32 * c.full(abs(H.P0) @ np.abs(vf))
    assert np.all(np.abs(gy - wy) <= ty)
    cons = np.ones(gy.size, bool)
    cons.reshape(-1, 3)[c.fn] = False
    assert np.all(gy[cons] == 0.0)
    # level products A_l x
    for l, shape in enumerate(H.shapes):
        fr = _lattice_free(shape)
        x = np.zeros(3 * np.prod(np.array(shape) + 1))
        x[fr] = rng.standard_normal(fr.size).astype(np.float32)
        xd = c.t(x, torch.float32)
        yd = torch.full_like(xd, 5.0)
        tm().tm_coarse_apply(ctx(), l, xd, yd)
        g = yd.double().cpu().numpy()
        X, Y, Z = shape
        K = torch.zeros(X * Y * Z * 576, dtype=torch.float32, device="cuda")
        tm().tm_coarse_cells(ctx(), l, K)
        Kh = np.abs(K.double().cpu().numpy().reshape(-1, 24, 24))
        scale = CO.assemble_cells(shape, Kh) @ np.abs(x[fr])
        w = H.A[l] @ x[fr]
        assert np.all(np.abs(g[fr] - w) <= 64 * U32 * scale + 4 * U32 * np.abs(w))
        fixed = np.ones(g.size, bool)
        fixed[fr] = False
        assert np.all(g[fixed] == 0.0)


@pytest.mark.parametrize("name", ["config1b", "small_truss", "truss_10x5x5_L1"])
@pytest.mark.parametrize("nu", [1, 2])
def test_vcycle_matches_the_oracle(name, nu):
    import torch
    c, rho, info, H = _setup(name)
    shape0 = H.shapes[0]
    fr = _lattice_free(shape0)
    rng = np.random.default_rng(40 + nu)
    b = np.zeros(3 * np.prod(np.array(shape0) + 1))
    b[fr] = rng.standard_normal(fr.size).astype(np.float32)
    bd = c.t(b, torch.float32)
    xd = torch.full_like(bd, 3.0)
    for _ in range(2):           # twice: nothing carries over between cycles
        tm().tm_coarse_vcycle(ctx(), bd, xd, nu)
        got = xd.double().cpu().numpy()
        want = H.vcycle(b[fr], nu)
        assert np.linalg.norm(got[fr] - want) <= 1e-4 * np.linalg.norm(want)
        fixed = np.ones(got.size, bool)
        fixed[fr] = False
        assert np.all(got[fixed] == 0.0)


@pytest.mark.parametrize("name,factor", [("config1b", 2.5), ("small_truss", 5.0), ("truss_10x5x5_L1", 2.5)])
def test_twolevel_solve_reaches_the_tolerance_in_fewer_iterations(name, factor):
    import torch
    P = tm()
    c = case(name)
    c.upload()
    rho = c.t(c.rho)
    f = c.t(c.full(c.f))
    u2 = torch.zeros_like(f)
    st2 = P.tm_pcg_solve(ctx(), rho, f, u2, rtol=1e-8, precision=P.TM_PREC_MIXED, precond=P.TM_PRECOND_TWOLEVEL)
    u1 = torch.zeros_like(f)
    st1 = P.tm_pcg_solve(ctx(), rho, f, u1, rtol=1e-8, precision=P.TM_PREC_MIXED)
    for u in (u2, u1):
        uf = c.free(u.cpu().numpy())
        assert np.linalg.norm(c.f - c.A @ uf) <= 1.0001e-8 * np.linalg.norm(c.f)
    assert st2["coarse_levels"] == len(CO.level_shapes(c.m))
    assert factor * st2["iterations"] <= st1["iterations"], (st2["iterations"], st1["iterations"])
    # close to the oracle's FP64 two-level PCG from the same start
    _, it_o, _ = CO.twolevel_pcg(c.m, c.A, c.f, rtol=1e-8, nu=1)
    assert st2["iterations"] <= 1.3 * it_o + 10, (st2["iterations"], it_o)
    # graph batches and plain launches give the same iterate bit for bit
    u3 = torch.zeros_like(f)
    st3 = P.tm_pcg_solve(ctx(), rho, f, u3, rtol=1e-8, precision=P.TM_PREC_MIXED, precond=P.TM_PRECOND_TWOLEVEL,
                         graphs=False)
    assert st3["iterations"] == st2["iterations"]
    assert torch.equal(u3, u2)


def test_twolevel_rejects_fp64_and_unknown_preconditioners():
    import torch
    P = tm()
    c = case("config1b")
    c.upload()
    rho = c.t(c.rho)
    f = c.t(c.full(c.f))
    u = torch.zeros_like(f)
    with pytest.raises(P.TmError) as e:
        P.tm_pcg_solve(ctx(), rho, f, u, precision=P.TM_PREC_FP64, precond=P.TM_PRECOND_TWOLEVEL)
    assert e.value.code == P.TM_EINVAL
    with pytest.raises(P.TmError) as e:
        P.tm_pcg_solve(ctx(), rho, f, u, precision=P.TM_PREC_MIXED, precond=7)
    assert e.value.code == P.TM_EINVAL
