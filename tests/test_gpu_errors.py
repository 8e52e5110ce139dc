"""Failure detection through status codes (no GPU fault is provoked: every failure is made
on the host side or is an argument the library rejects before launching)."""
import numpy as np
import pytest

from tests.gpu_common import case, ctx, tm

pytestmark = pytest.mark.gpu


def test_calls_before_a_mesh_report_state_error():
    import torch
    P = tm()
    c = P.tm_create(0, stream=torch.cuda.current_stream())
    c.info = {"Ne": 1, "Nn": 1}
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TmError) as ei:
        P.tm_apply_K(c, torch.zeros(1, dtype=torch.float64, device="cuda"), x, x.clone())
    assert ei.value.code == P.TM_ESTATE
    P.tm_destroy(c)


def test_invalid_mesh_is_rejected_by_upload():
    P = tm()
    import workloads as W
    dom = W.Domain(2, 1, 1, 2, 1.0)
    one = W.refine(dom, W.uniform_leaves(dom), [True, False])
    bad = W.refine(dom, one, (one[:, 3] == 1) & (one[:, 0] == 2) & (one[:, 1] == 0) & (one[:, 2] == 0))
    with pytest.raises(P.TmError) as ei:
        P.tm_mesh_upload(ctx(), 2, 1, 1, 2, 1.0, bad)
    assert ei.value.code == P.TM_EINVAL
    assert "balanced" in str(ei.value)


def test_solver_status_codes():
    import torch
    P = tm()
    c = case("config1")
    c.upload()
    w = c.w
    f = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device=c.dev)
    P.tm_build_rhs(ctx(), w.load_nodes, w.load_comp, w.load_val, f)
    # max_iter reached: TM_ENOTCONVERGED with the stats of the last iterate
    u = torch.zeros_like(f)
    st = P.tm_pcg_solve(ctx(), c.t(c.rho), f, u, rtol=1e-12, max_iter=5, precision=0, raise_on_error=False)
    assert st["status"] == P.TM_ENOTCONVERGED
    assert st["iterations"] == 5 and st["rel_residual"] > 1e-12
    # a NaN in the design reaches a reduction: TM_ENONFINITE, no hang
    rho = c.rho.copy()
    rho[7] = np.nan
    for prec in (0, 1):
        u = torch.zeros_like(f)
        st = P.tm_pcg_solve(ctx(), c.t(rho), f, u, rtol=1e-8, max_iter=1000, precision=prec, raise_on_error=False)
        assert st["status"] == P.TM_ENONFINITE
    # zero load: u = 0 at once
    u = torch.ones_like(f)
    st = P.tm_pcg_solve(ctx(), c.t(c.rho), torch.zeros_like(f), u, rtol=1e-8)
    assert st["status"] == 0 and float(u.abs().max()) == 0.0


def test_argument_errors():
    import torch
    P = tm()
    c = case("config1")
    c.upload()
    rho = c.t(c.rho)
    out = torch.zeros_like(rho)
    with pytest.raises(P.TmError) as ei:
        P.tm_filter(ctx(), rho, rho, 10.0, 0, out)          # radius beyond the supported box
    assert ei.value.code == P.TM_EINVAL
    with pytest.raises(P.TmError) as ei:
        P.tm_filter(ctx(), rho, rho, 0.1, 7, out)           # unknown mode
    assert ei.value.code == P.TM_EINVAL
    with pytest.raises(P.TmError) as ei:
        P.tm_oc_update(ctx(), rho, -rho, 1.5, 0.2, 0.5, 1e-3, out)
    assert ei.value.code == P.TM_EINVAL
    f = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device=c.dev)
    with pytest.raises(P.TmError) as ei:
        P.tm_build_rhs(ctx(), [[100, 0, 0]], [2], [-1.0], f)  # not a node of this mesh
    assert ei.value.code == P.TM_EINVAL
    with pytest.raises(ValueError):
        P.tm_apply_K(ctx(), rho, f[:-3], f)                 # wrong length (binding check)
