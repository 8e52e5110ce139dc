"""Parity of every C-ABI entry point with the FP64 oracle on the same seeded inputs.

Tolerances (stated per test) follow from the arithmetic:
* integer tables: bit-exact;
* operator: the library evaluates each entry of A x in a different order than the
  oracle's assembled CSR (symmetry-adapted element product, per-node slot sums,
  partial sums of block-shared nodes), so entry i may differ by a small multiple of the unit roundoff u
  times (|A| |x|)_i, the standard bound for a reordered sum of products; the
  multiple 256 covers the ~60 operations on any path through the element
  kernel and the <= 16 contributions per node;
* solves: the residual of the returned u measured with the oracle's A in FP64.
"""
import numpy as np
import pytest

from tests.gpu_common import U32, U64, case, ctx, tm

pytestmark = pytest.mark.gpu

CASES = ["config1", "config1b", "small_truss"]


@pytest.fixture(scope="module", params=CASES)
def up(request):
    c = case(request.param)
    c.info = c.upload()
    return c


def test_uploaded_tables_bit_exact(up):
    t = tm().tm_mesh_tables(ctx())
    m = up.m
    assert np.array_equal(t["perm"], m.perm)
    assert np.array_equal(t["node_xyz"], m.nodes)
    assert np.array_equal(t["conn"], m.conn)
    assert np.array_equal(t["hang_node"], m.hanging_ids())


def _abs_bound(c, x_free):
    return abs(c.A) @ np.abs(x_free)


def test_apply_fp64_matches_assembled_operator(up):
    import torch
    rng = np.random.default_rng(11)
    x = rng.standard_normal(up.A.shape[0])
    y_ref = up.A @ x
    xd = up.t(up.full(x))
    # garbage at constrained DOFs must be ignored
    xd_dirty = xd.clone()
    cons = torch.ones(xd.numel(), dtype=torch.bool, device=xd.device)
    cons.view(-1, 3)[torch.as_tensor(up.fn, device=xd.device)] = False
    xd_dirty[cons] = 123.0
    yd = torch.full_like(xd, 7.0)
    rho = up.t(up.rho)
    tm().tm_apply_K(ctx(), rho, xd_dirty, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.all(y[cons.cpu().numpy()] == 0.0)
    err = np.abs(up.free(y) - y_ref)
    assert np.all(err <= 256 * U64 * _abs_bound(up, x))


def test_apply_fp32_matches_assembled_operator(up):
    import torch
    rng = np.random.default_rng(12)
    x = rng.standard_normal(up.A.shape[0]).astype(np.float32).astype(np.float64)
    y_ref = up.A @ x
    xd = up.t(up.full(x), torch.float32)
    yd = torch.zeros_like(xd)
    tm().tm_apply_K_f32(ctx(), up.t(up.rho), xd, yd)
    torch.cuda.synchronize()
    err = np.abs(up.free(yd.double().cpu().numpy()) - y_ref)
    # FP32 coefficients and arithmetic: same bound with u = 2^-23
    assert np.all(err <= 256 * U32 * _abs_bound(up, x))


def test_apply_is_deterministic(up):
    import torch
    rng = np.random.default_rng(13)
    xd = up.t(up.full(rng.standard_normal(up.A.shape[0])))
    rho = up.t(up.rho)
    y1, y2 = torch.zeros_like(xd), torch.zeros_like(xd)
    tm().tm_apply_K(ctx(), rho, xd, y1)
    tm().tm_apply_K(ctx(), rho, xd, y2)
    assert torch.equal(y1, y2)


def test_jacobi_diagonal(up):
    import torch
    d = torch.zeros(3 * up.m.Nn, dtype=torch.float64, device=up.dev)
    tm().tm_jacobi_diag(ctx(), up.t(up.rho), d)
    ref = up.A.diagonal()
    got = up.free(d.cpu().numpy())
    assert np.allclose(got, ref, rtol=64 * U64, atol=0)


def test_rhs(up):
    import torch
    f = torch.full((3 * up.m.Nn,), 5.0, dtype=torch.float64, device=up.dev)
    w = up.w
    tm().tm_build_rhs(ctx(), w.load_nodes, w.load_comp, w.load_val, f)
    got = f.cpu().numpy()
    assert np.array_equal(up.free(got), up.f)
    assert np.count_nonzero(got) == np.count_nonzero(up.f)


def test_expand_matches_constraint_matrix(up):
    import torch
    rng = np.random.default_rng(14)
    u = rng.standard_normal(up.A.shape[0])
    ud = up.t(up.full(u))
    uf = torch.zeros_like(ud)
    tm().tm_expand(ctx(), ud, uf)
    ref = up.C @ u
    assert np.allclose(uf.cpu().numpy(), ref, rtol=4 * U64, atol=0)


def _solve(up, precision, rtol, warm=None):
    import torch
    f = torch.zeros(3 * up.m.Nn, dtype=torch.float64, device=up.dev)
    w = up.w
    tm().tm_build_rhs(ctx(), w.load_nodes, w.load_comp, w.load_val, f)
    u = torch.zeros_like(f) if warm is None else up.t(up.full(warm))
    st = tm().tm_pcg_solve(ctx(), up.t(up.rho), f, u, rtol=rtol, max_iter=200000, precision=precision)
    return up.free(u.cpu().numpy()), st


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_residual_in_oracle_operator(up, precision):
    """Parity criterion for solves: ||f - A u|| / ||f|| <= 1e-8 with the oracle's A in FP64."""
    u, st = _solve(up, precision, 1e-8)
    rel = np.linalg.norm(up.f - up.A @ u) / np.linalg.norm(up.f)
    assert st["status"] == 0
    assert rel <= 1e-8 * (1 + 1e-3)
    assert abs(st["rel_residual"] - rel) <= 1e-3 * rel + 1e-14


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_solution_and_compliance_against_direct(up, precision):
    """Tight solve (1e-12): u within 1e-8 of the oracle's direct solution in the energy
    norm, and compliance within 1e-8."""
    ud = up.direct()
    u, st = _solve(up, precision, 1e-12)
    e = u - ud
    energy_err = np.sqrt(abs(e @ (up.A @ e))) / np.sqrt(ud @ (up.A @ ud))
    assert energy_err <= 1e-8
    c_ref = up.f @ ud
    assert abs(up.f @ u - c_ref) <= 1e-8 * abs(c_ref)


def test_sensitivity_and_compliance(up):
    import torch
    from oracle import topopt as T
    ud = up.direct()
    uf = up.C @ ud
    w = up.w
    ref = T.sensitivity(up.m, up.rho, uf, w.E0, w.Emin, w.nu, w.penal)
    dc = torch.zeros(up.m.Ne, dtype=torch.float64, device=up.dev)
    comp = tm().tm_sensitivity(ctx(), up.t(up.rho), up.t(uf), dc)
    got = dc.cpu().numpy()
    # u_e^T K0 u_e is a sum of 576 products whose magnitudes |u_e|^T |K0| |u_e| can exceed the
    # result by orders of magnitude (near-rigid element motion): both sides' rounding is bounded
    # by a small multiple of u times that sum.
    from oracle import fem as F
    K0 = F.reference_stiffness(w.nu)
    ue = np.abs(uf[F.element_dofs(up.m)])
    mag = np.einsum("ei,ij,ej->e", ue, np.abs(K0), ue)
    scale = w.penal * up.rho ** (w.penal - 1) * (w.E0 - w.Emin) * up.m.h * mag
    assert np.all(np.abs(got - ref) <= 256 * U64 * scale)
    c_ref = T.compliance_by_elements(up.m, up.rho, uf, w.E0, w.Emin, w.nu, w.penal)
    cscale = np.sum(F.young(up.rho, w.E0, w.Emin, w.penal) * up.m.h * mag)
    assert abs(comp - c_ref) <= 256 * U64 * cscale
    assert comp == pytest.approx(up.f @ ud, rel=1e-9)


@pytest.mark.parametrize("mode", [0, 1])
def test_filter(up, mode):
    import torch
    from oracle import topopt as T
    rng = np.random.default_rng(15)
    x = -rng.uniform(0, 1, up.m.Ne)
    rmin = up.w.r_min
    ref = T.sensitivity_filter(up.m, up.rho, x, rmin) if mode == 0 else T.density_filter(up.m, x, rmin)
    out = torch.zeros(up.m.Ne, dtype=torch.float64, device=up.dev)
    tm().tm_filter(ctx(), up.t(up.rho), up.t(x), rmin, mode, out)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=0)


def test_oc_update(up):
    import torch
    from oracle import topopt as T
    rng = np.random.default_rng(16)
    dc = -rng.uniform(1e-6, 1, up.m.Ne) * up.m.volume
    V = up.m.volume
    volfrac = float(np.sum(up.rho * V) / V.sum())
    rho_new = torch.zeros(up.m.Ne, dtype=torch.float64, device=up.dev)
    change = tm().tm_oc_update(ctx(), up.t(up.rho), up.t(dc), volfrac, 0.2, 0.5, 1e-3, rho_new)
    got = rho_new.cpu().numpy()
    ref, ref_change, lam = T.oc_update(up.rho, dc, V, volfrac * V.sum(), 0.2, 0.5, 1e-3)
    assert abs(np.sum(got * V) - volfrac * V.sum()) <= 1e-10 * V.sum()
    assert got.min() >= 1e-3 and got.max() <= 1.0
    assert np.all(np.abs(got - up.rho) <= 0.2 + 1e-15)
    # both bisect lambda to a 1e-12 relative bracket: designs agree to ~1e-12
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)
    assert change == pytest.approx(ref_change, rel=1e-9, abs=1e-12)
