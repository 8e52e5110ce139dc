"""The autotuner (paper_1009_4975_gb300.autotune): it times every candidate with the library's
own solves, keeps the fastest, caches the choice per mesh, and its choice solves to the same
tolerance."""
import numpy as np
import pytest

from tests.gpu_common import case, ctx, tm

pytestmark = pytest.mark.gpu


def test_autotuner_picks_the_fastest_candidate_and_caches_it():
    import torch
    from paper_1009_4975_gb300 import autotune as AT
    P = tm()
    c = case("config1b")
    c.upload()
    rho = c.t(c.rho)
    f = c.t(c.full(c.f))
    u0 = torch.zeros_like(f)
    best = AT.tune_solve(ctx(), rho, f, u0, check_every=(8, 32), smooth_sweeps=(1, 2), repeats=2, refresh=True)
    assert len(best["table"]) == 4
    assert best["seconds"] == min(r["seconds"] for r in best["table"])
    assert AT.tune_solve(ctx(), rho, f, u0) is best                     # cached for this mesh
    u = u0.clone()
    st = P.tm_pcg_solve(ctx(), rho, f, u, rtol=1e-8, precision=P.TM_PREC_MIXED, precond=P.TM_PRECOND_TWOLEVEL,
                        smooth_sweeps=best["smooth_sweeps"], check_every=best["check_every"])
    uf = c.free(u.cpu().numpy())
    assert np.linalg.norm(c.f - c.A @ uf) <= 1.0001e-8 * np.linalg.norm(c.f)
    assert float(u0.abs().max()) == 0.0                                 # the start is not modified
    F = torch.stack([f, -f, 0.5 * f]).contiguous()
    bm = AT.tune_multi(ctx(), rho, F, groups=(4, 2, 1), repeats=1, refresh=True, precond=P.TM_PRECOND_TWOLEVEL)
    assert {r["group"] for r in bm["table"]} == {2, 1}
    assert bm["group"] in (1, 2)
