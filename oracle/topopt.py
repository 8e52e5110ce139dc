"""Oracle optimisation steps: compliance, sensitivities, filters and OC
(paper Sec. 3 Eq. 1-2, Sec. 6 Eq. 3-5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings where the paper names a step without a formula:

* Sensitivity (Sec. 3): for compliance ``c = f^T u`` with ``K(rho) u = f`` the
  adjoint is u itself, so ``dc/drho_e = -u_e^T (dK_e/drho_e) u_e =
  -p rho_e^(p-1) (E0 - Emin) h_e u_e^T K0 u_e`` with ``u_e`` the element's 24
  corner values of ``u_full = C u``.
* OC (Sec. 3): the standard optimality-criteria heuristic,
  ``rho_new = clamp(rho * (max(-dc, 0) / (lambda V_e))^eta, max(rho_min, rho - m),
  min(1, rho + m))`` with lambda found by bisection so that
  ``sum rho_new V_e = volfrac * |Omega|``.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .fem import element_dofs, reference_stiffness, young
from .mesh import Mesh


def element_energy(mesh: Mesh, u_full: np.ndarray, nu: float) -> np.ndarray:
    """u_e^T K0 u_e per element (unit-cube, E = 1 stiffness)."""
    K0 = reference_stiffness(nu)
    ue = np.asarray(u_full)[element_dofs(mesh)]          # (Ne, 24)
    return np.einsum("ei,ij,ej->e", ue, K0, ue)


def compliance(f: np.ndarray, u: np.ndarray) -> float:
    """c = f^T u (Eq. 1)."""
    return float(np.dot(f, u))


def compliance_by_elements(mesh: Mesh, rho, u_full, E0, Emin, nu, penal) -> float:
    return float(np.sum(young(rho, E0, Emin, penal) * mesh.h * element_energy(mesh, u_full, nu)))


def sensitivity(mesh: Mesh, rho, u_full, E0, Emin, nu, penal) -> np.ndarray:
    rho = np.asarray(rho, np.float64)
    return -penal * rho ** (penal - 1) * (E0 - Emin) * mesh.h * element_energy(mesh, u_full, nu)


def filter_pairs(mesh: Mesh, rmin: float):
    """All (e, d) with centre distance < rmin, including e = d, and H_de = rmin - dist (Eq. 4)."""
    c = mesh.centres
    tree = cKDTree(c)
    D = tree.sparse_distance_matrix(tree, rmin, output_type="coo_matrix")
    e, d, dist = D.row, D.col, D.data
    keep = (dist < rmin) & (e != d)
    e, d, dist = e[keep], d[keep], dist[keep]
    # the self pair (distance 0) is added explicitly, once
    self_ = np.arange(mesh.Ne)
    e = np.concatenate([e, self_])
    d = np.concatenate([d, self_])
    H = np.concatenate([rmin - dist, np.full(mesh.Ne, rmin)])
    return e, d, H


def filter_pairs_bruteforce(mesh: Mesh, rmin: float):
    c = mesh.centres
    out_e, out_d, out_H = [], [], []
    for e in range(mesh.Ne):
        for d in range(mesh.Ne):
            dist = np.sqrt(np.sum((c[e] - c[d]) ** 2))
            H = max(rmin - dist, 0.0)
            if H > 0:
                out_e.append(e)
                out_d.append(d)
                out_H.append(H)
    return np.array(out_e), np.array(out_d), np.array(out_H)


def sensitivity_filter(mesh: Mesh, rho, dc, rmin, pairs=None) -> np.ndarray:
    """Eq. 5: dc_hat_e = sum_d rho_d H_de V_d dc_d / (rho_e sum_d H_de V_d)."""
    e, d, H = filter_pairs(mesh, rmin) if pairs is None else pairs
    V = mesh.volume
    rho = np.asarray(rho, np.float64)
    w = H * V[d]
    num = np.bincount(e, weights=w * rho[d] * np.asarray(dc)[d], minlength=mesh.Ne)
    den = np.bincount(e, weights=w, minlength=mesh.Ne)
    return num / (rho * den)


def sigmund_filter(mesh: Mesh, rho, dc, rmin, pairs=None) -> np.ndarray:
    """Eq. 3 (no volume weights), for the uniform-mesh special case."""
    e, d, H = filter_pairs(mesh, rmin) if pairs is None else pairs
    rho = np.asarray(rho, np.float64)
    num = np.bincount(e, weights=H * rho[d] * np.asarray(dc)[d], minlength=mesh.Ne)
    den = np.bincount(e, weights=H, minlength=mesh.Ne)
    return num / (rho * den)


def density_filter(mesh: Mesh, x, rmin, pairs=None) -> np.ndarray:
    """Volume-weighted density filter: sum_d H_de V_d x_d / sum_d H_de V_d."""
    e, d, H = filter_pairs(mesh, rmin) if pairs is None else pairs
    w = H * mesh.volume[d]
    num = np.bincount(e, weights=w * np.asarray(x)[d], minlength=mesh.Ne)
    den = np.bincount(e, weights=w, minlength=mesh.Ne)
    return num / den


def oc_update(rho, dc, V, volfrac_volume, move=0.2, eta=0.5, rho_min=1e-3, rtol=1e-12, max_iter=200):
    """Bisection on lambda until the bracket is relatively smaller than rtol.

    Returns (rho_new, max |rho_new - rho|, lambda)."""
    rho = np.asarray(rho, np.float64)
    V = np.asarray(V, np.float64)
    g = np.maximum(-np.asarray(dc, np.float64), 0.0)
    lo_b = np.maximum(rho_min, rho - move)
    hi_b = np.minimum(1.0, rho + move)

    def update(lam):
        return np.clip(rho * (g / (lam * V)) ** eta, lo_b, hi_b)

    l1, l2 = 0.0, 1e9 * max(g.max(), 1e-300) / V.min()
    for _ in range(max_iter):
        lm = 0.5 * (l1 + l2)
        if np.sum(update(lm) * V) > volfrac_volume:
            l1 = lm
        else:
            l2 = lm
        if (l2 - l1) <= rtol * (l1 + l2):
            break
    lm = 0.5 * (l1 + l2)
    new = update(lm)
    return new, float(np.max(np.abs(new - rho))), lm
