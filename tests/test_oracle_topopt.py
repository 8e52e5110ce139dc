"""Pins for compliance, sensitivities, filters (paper Eq. 1, 3-5) and the OC update."""
import numpy as np
import pytest

import workloads as W
from oracle import fem as F
from oracle import mesh as M
from oracle import solve as S
from oracle import topopt as T

E0, EMIN, NU, P = 1.0, 1e-9, 0.3, 3.0


def _mesh(w):
    d = w.dom
    return M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)


def _solve(m, w, rho):
    A, f, C = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val, E0, EMIN, NU, P)
    u = S.direct(A, f)
    return A, f, C, u


def test_sensitivities_match_central_differences_of_compliance():
    w = W.config1()
    m = _mesh(w)
    rho = 0.3 + 0.7 * w.rho[m.perm]
    A, f, C, u = _solve(m, w, rho)
    dc = T.sensitivity(m, rho, C @ u, E0, EMIN, NU, P)
    assert (dc <= 0).all()
    h = 1e-5
    worst = 0.0
    for e in range(0, m.Ne, 23):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        cp = f @ _solve(m, w, rp)[3]
        cm = f @ _solve(m, w, rm)[3]
        worst = max(worst, abs((cp - cm) / (2 * h) - dc[e]) / np.abs(dc).max())
    assert worst < 1e-6


def test_compliance_equals_element_energy_sum():
    w = W.config1()
    m = _mesh(w)
    rho = w.rho[m.perm]
    A, f, C, u = _solve(m, w, rho)
    c1 = T.compliance(f, u)
    c2 = T.compliance_by_elements(m, rho, C @ u, E0, EMIN, NU, P)
    assert abs(c1 - c2) <= 1e-9 * c1
    # and c = -sum rho_e dc_e / p when Emin = 0 (homogeneity of degree p in rho)
    A0, f0, C0 = F.reduced_system(m, rho, w.load_nodes, w.load_comp, w.load_val, E0, 0.0, NU, P)
    u0 = S.direct(A0, f0)
    dc0 = T.sensitivity(m, rho, C0 @ u0, E0, 0.0, NU, P)
    assert abs(-np.sum(rho * dc0) / P - f0 @ u0) <= 1e-8 * (f0 @ u0)


def test_filter_pairs_match_bruteforce():
    w = W.config1()
    m = _mesh(w)
    for rmin in (w.r_min, 0.3):
        e1, d1, H1 = T.filter_pairs(m, rmin)
        e2, d2, H2 = T.filter_pairs_bruteforce(m, rmin)
        a = sorted(zip(e1.tolist(), d1.tolist()))
        b = sorted(zip(e2.tolist(), d2.tolist()))
        assert a == b
        o1 = np.lexsort((d1, e1))
        o2 = np.lexsort((d2, e2))
        assert np.allclose(H1[o1], H2[o2], rtol=0, atol=1e-15)


def test_volume_weighted_filter_reduces_to_sigmund_on_uniform_mesh():
    dom = W.Domain(6, 3, 3, 0, 1.0 / 3.0)
    m = M.build_mesh(6, 3, 3, 0, dom.h0, W.uniform_leaves(dom))
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.01, 1, m.Ne)
    dc = -rng.uniform(0, 1, m.Ne)
    for rmin in (0.5, 0.8):
        a = T.sensitivity_filter(m, rho, dc, rmin)
        b = T.sigmund_filter(m, rho, dc, rmin)
        assert np.allclose(a, b, rtol=1e-14, atol=0)


def test_filter_deactivates_below_smallest_element():
    """No neighbours within rmin (paper Sec. 6): the filter is the identity."""
    w = W.config1b()
    m = _mesh(w)
    rng = np.random.default_rng(4)
    dc = -rng.uniform(0, 1, m.Ne)
    rho = m.volume * 0 + rng.uniform(0.01, 1, m.Ne)
    out = T.sensitivity_filter(m, rho, dc, 0.9 * w.dom.h_min)
    assert np.allclose(out, dc, rtol=1e-15, atol=0)
    assert np.allclose(T.density_filter(m, rho, 0.9 * w.dom.h_min), rho, rtol=1e-15, atol=0)


def test_filter_of_constant_field():
    w = W.config1b()
    m = _mesh(w)
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.01, 1, m.Ne)
    rmin = w.r_min
    e, d, H = T.filter_pairs(m, rmin)
    out = T.sensitivity_filter(m, rho, np.full(m.Ne, -2.0), rmin, pairs=(e, d, H))
    w_ = H * m.volume[d]
    expect = -2.0 * np.bincount(e, weights=w_ * rho[d], minlength=m.Ne) / (rho * np.bincount(e, weights=w_, minlength=m.Ne))
    assert np.allclose(out, expect, rtol=1e-14)
    # density filter preserves constants exactly up to rounding
    assert np.allclose(T.density_filter(m, np.full(m.Ne, 0.37), rmin), 0.37, rtol=1e-14)
    # and preserves the volume-weighted mean only approximately; it is a convex average
    x = rng.uniform(0, 1, m.Ne)
    fx = T.density_filter(m, x, rmin)
    assert fx.min() >= x.min() - 1e-15 and fx.max() <= x.max() + 1e-15


def test_oc_update_meets_volume_bounds_and_move_limits():
    w = W.config1b()
    m = _mesh(w)
    rng = np.random.default_rng(6)
    rho = rng.uniform(0.001, 1, m.Ne)
    dc = -rng.uniform(1e-6, 1, m.Ne)
    V = m.volume
    target = 0.45 * V.sum()          # reachable within the move limit from a U(0,1) design
    new, change, lam = T.oc_update(rho, dc, V, target, move=0.2, eta=0.5, rho_min=1e-3)
    assert abs(np.sum(new * V) - target) <= 1e-11 * V.sum()
    assert new.min() >= 1e-3 and new.max() <= 1.0
    assert (np.abs(new - rho) <= 0.2 + 1e-15).all()
    assert change == pytest.approx(np.abs(new - rho).max())
    # the update formula holds for an interior element
    B = (-dc / (lam * V)) ** 0.5
    inner = (rho * B > np.maximum(1e-3, rho - 0.2)) & (rho * B < np.minimum(1.0, rho + 0.2))
    assert inner.sum() > 10
    assert np.allclose(new[inner], (rho * B)[inner], rtol=1e-14)


def test_oc_fixed_point():
    """When -dc / V is uniform and the design already meets the volume, OC returns it unchanged."""
    dom = W.Domain(4, 2, 2, 0, 0.5)
    m = M.build_mesh(4, 2, 2, 0, 0.5, W.uniform_leaves(dom))
    V = m.volume
    rho = np.full(m.Ne, 0.4)
    dc = -3.0 * V
    new, change, lam = T.oc_update(rho, dc, V, 0.4 * V.sum())
    assert np.allclose(new, rho, rtol=1e-11)
    assert lam == pytest.approx(3.0, rel=1e-10)


def test_filter_worked_example_on_mixed_sizes():
    """Hand-worked Eq. 5 on a mesh with two element sizes (fixture derivation in the file)."""
    import os
    dom = W.Domain(2, 1, 1, 1, 1.0)
    leaves = W.refine(dom, W.uniform_leaves(dom), np.array([True, False]))
    m = M.build_mesh(2, 1, 1, 1, 1.0, leaves, dirichlet_faces=0)
    dc = np.where(m.leaves[:, 3] == 0, -2.0, -1.0)
    out = T.sensitivity_filter(m, np.ones(m.Ne), dc, 0.9)
    path = os.path.join(os.path.dirname(__file__), "golden", "filter_2x1x1_L1.txt")
    rows = [l.split("|") for l in open(path) if l.strip() and not l.startswith("#")]
    for c, v in rows:
        e = int(np.argmin(np.abs(m.centres - np.array([float(t) for t in c.split()])).sum(axis=1)))
        assert out[e] == pytest.approx(float(v), rel=1e-14)
