"""The OC update's lambda search and the filter's tabulated weights beyond the defaults of
`test_gpu_parity.py`, against the oracle.

* OC (Sec. 3): the library finds lambda by a safeguarded Newton search on the piecewise linear
  volume, the oracle by bisection; both stop at a relative lambda bracket of 1e-12, so the
  designs agree to 1e-9.  Cases: eta = 0.3 (the pow() path instead of the square root), a
  volume target that puts most elements on their move limits, one near the upper bound of the
  total volume, and a sensitivity field with zeros (elements whose factor is 0 stay at their
  lower bound for every lambda).
* Filter (Eq. 5 and the density filter): the weight of a neighbour depends only on its level
  and the exact integer squared distance of the centres in half finest cells; radii of 4 finest
  cells (the largest the library takes), 2.3 and 0.9 (below the smallest centre distance: only
  the element itself, the identity).  A radius equal to a centre distance (1 finest cell) is left
  out: the library excludes such ties exactly (dist < rmin in integers), while the oracle's
  floating-point distances put some of them just inside the radius with weights of order 1e-16.
  One-signed inputs as in the method, and the tolerance of the default radius, rtol 1e-13.
"""
import numpy as np
import pytest

from tests.gpu_common import case, ctx, tm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def truss():
    c = case("small_truss")
    c.upload()
    return c


def _oc(c, dc, volfrac, move, eta, rho_min):
    import torch
    from oracle import topopt as T
    V = c.m.volume
    rho_new = torch.zeros(c.m.Ne, dtype=torch.float64, device=c.dev)
    change = tm().tm_oc_update(ctx(), c.t(c.rho), c.t(dc), volfrac, move, eta, rho_min, rho_new)
    got = rho_new.cpu().numpy()
    ref, ref_change, _ = T.oc_update(c.rho, dc, V, volfrac * V.sum(), move, eta, rho_min)
    return got, change, ref, ref_change, V


@pytest.mark.parametrize("eta,volscale,zeros", [(0.3, 1.0, False), (0.5, 0.75, False), (0.5, 1.25, False),
                                                (0.5, 1.0, True)])
def test_oc_lambda_search_against_bisection(truss, eta, volscale, zeros):
    c = truss
    rng = np.random.default_rng(31)
    dc = -rng.uniform(1e-6, 1, c.m.Ne) * c.m.volume
    if zeros:
        dc[rng.random(c.m.Ne) < 0.2] = 0.0
    V = c.m.volume
    volfrac = min(0.99, volscale * float(np.sum(c.rho * V) / V.sum()))
    got, change, ref, ref_change, V = _oc(c, dc, volfrac, 0.2, eta, 1e-3)
    assert abs(np.sum(got * V) - volfrac * V.sum()) <= 1e-10 * V.sum()
    assert got.min() >= 1e-3 and got.max() <= 1.0
    assert np.all(np.abs(got - c.rho) <= 0.2 + 1e-15)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)
    assert change == pytest.approx(ref_change, rel=1e-9, abs=1e-12)
    if volscale != 1.0:   # the target moves many elements onto a move limit
        lo, hi = np.maximum(1e-3, c.rho - 0.2), np.minimum(1.0, c.rho + 0.2)
        assert np.mean((got == lo) | (got == hi)) > 0.2


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("cells", [4.0, 2.3, 0.9])
def test_filter_radii(truss, mode, cells):
    import torch
    from oracle import topopt as T
    c = truss
    hmin = c.w.dom.h0 / (1 << c.w.dom.L)
    rmin = cells * hmin
    # one-signed inputs as in the method (dc <= 0, densities > 0): every output is a weighted
    # mean of same-signed values, so a relative bound holds entrywise
    rng = np.random.default_rng(32)
    x = -rng.uniform(0, 1, c.m.Ne) if mode == 0 else rng.uniform(1e-3, 1, c.m.Ne)
    ref = T.sensitivity_filter(c.m, c.rho, x, rmin) if mode == 0 else T.density_filter(c.m, x, rmin)
    out = torch.zeros(c.m.Ne, dtype=torch.float64, device=c.dev)
    tm().tm_filter(ctx(), c.t(c.rho), c.t(x), rmin, mode, out)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=0)
