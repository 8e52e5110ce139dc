"""The autotuner's choice and cache (paper_1009_4975_gb300.autotune) on the host: the library's
solve entry points are replaced by stand-ins whose cost is known (a sleep per call), so the test
needs no GPU.  The autotuner must time every candidate, keep the fastest, cache the choice per mesh
and kind, and time again on refresh.  `test_gpu_autotune.py` runs it on the library itself."""
import types

import pytest
import torch

from paper_1009_4975_gb300 import autotune as AT


class _Ctx:
    def __init__(self, ne):
        self.info = {"Ne": ne, "Nn": 2 * ne, "n_hanging": 0, "n_blocks": 1}


@pytest.fixture
def fake(monkeypatch):
    calls = []
    cost = {}

    def solve(ctx, rho, f, u, **kw):
        calls.append(("solve", kw["check_every"], kw["smooth_sweeps"]))
        import time
        time.sleep(cost.get(("solve", kw["check_every"], kw["smooth_sweeps"]), 0.01))

    def solve_multi(ctx, rho, F, U, **kw):
        calls.append(("multi", int(F.shape[0])))
        import time
        time.sleep(cost.get(("multi", int(F.shape[0])), 0.01))

    monkeypatch.setattr(AT, "T", types.SimpleNamespace(tm_pcg_solve=solve, tm_pcg_solve_multi=solve_multi,
                                                       TM_PREC_MIXED=1, TM_PRECOND_TWOLEVEL=1))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(AT, "_cache", {})
    return calls, cost


def test_solve_tuning_picks_the_fastest_and_caches_it(fake):
    calls, cost = fake
    cost[("solve", 16, 1)] = 0.0005            # the one fast candidate
    ctx, x = _Ctx(1000), torch.zeros(3)
    best = AT.tune_solve(ctx, x, x, x, repeats=3)
    assert (best["check_every"], best["smooth_sweeps"]) == (16, 1)
    # every candidate: one warm-up solve and `repeats` timed ones
    assert len(best["table"]) == 6 and len(calls) == 6 * 4
    assert AT.tune_solve(ctx, x, x, x, repeats=3) is best and len(calls) == 24      # cached
    assert AT.tune_solve(_Ctx(1001), x, x, x, repeats=1)["check_every"] == 16      # another mesh
    assert len(calls) == 24 + 6 * 2
    cost[("solve", 16, 1)] = 0.01
    cost[("solve", 32, 2)] = 0.0005
    again = AT.tune_solve(ctx, x, x, x, repeats=1, refresh=True)
    assert (again["check_every"], again["smooth_sweeps"]) == (32, 2)


def test_multi_tuning_keeps_groups_within_the_cases_and_prefers_larger_ones(fake):
    calls, cost = fake
    ctx = _Ctx(500)
    x = torch.zeros(3)
    F = torch.zeros((6, 9))
    # every group size costs the same per call: one call per group, so the largest group wins
    best = AT.tune_multi(ctx, x, F, repeats=1)
    assert [r["group"] for r in best["table"]] == [4, 2, 1]        # 8 > 6 cases is skipped
    assert best["group"] == 4
    # calls per candidate (warm-up + 1 timed): ceil(6 / g) each
    assert sum(1 for c in calls if c[0] == "multi") == 2 * (2 + 3 + 6)
    # a different case count is a different cache entry
    assert AT.tune_multi(ctx, x, torch.zeros((2, 9)), repeats=1)["group"] == 2
