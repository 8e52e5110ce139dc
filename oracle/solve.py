"""Oracle linear solvers for the reduced system A u = f (paper Sec. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``direct`` -- sparse LU of A (SciPy SuperLU), the reference solution.
* ``dense_cholesky`` -- a textbook column Cholesky, written out, for tiny systems
  (an independent check on the sparse factorisation).
* ``twolevel_pcg`` -- PCG with the additive two-level preconditioner
  M^-1 = D^-1 + P (P^T A P)^-1 P^T (Jacobi plus a Galerkin coarse correction on a
  coarse space given by a prolongation P, e.g. ``grid_prolongation``); no paper
  counterpart: the coarse-grid correction of the learned part's extension.
* ``VCycle`` -- an approximate coarse solve: a V-cycle over uniform cell-centred grids
  (Galerkin operators, trilinear transfers, symmetric damped-Jacobi smoothing with
  omega = 1 / lambda_max(D^-1 A) per level, a direct solve on the coarsest grid), a
  fixed SPD operator that can replace (P^T A P)^-1 in the two-level preconditioner.
* ``jacobi_pcg`` -- preconditioned CG with the diagonal of A as preconditioner.
  Diagonal (Jacobi) preconditioning is the symmetric rescaling
  ``D^{-1/2} A D^{-1/2}`` of Sec. 5 applied implicitly: CG on the rescaled
  system and Jacobi-PCG on A produce the same iterates.  This is also the CPU
  baseline the bench times.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def direct(A: sp.spmatrix, f: np.ndarray) -> np.ndarray:
    return spla.splu(A.tocsc()).solve(np.asarray(f, np.float64))


def dense_cholesky(A: np.ndarray) -> np.ndarray:
    A = np.array(A, np.float64)
    n = A.shape[0]
    Lm = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - Lm[j, :j] @ Lm[j, :j]
        if s <= 0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        Lm[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            Lm[i, j] = (A[i, j] - Lm[i, :j] @ Lm[j, :j]) / Lm[j, j]
    return Lm


def cholesky_solve(Lm: np.ndarray, f: np.ndarray) -> np.ndarray:
    n = Lm.shape[0]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (f[i] - Lm[i, :i] @ y[:i]) / Lm[i, i]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - Lm[i + 1:, i] @ x[i + 1:]) / Lm[i, i]
    return x


def relative_residual(A, u, f) -> float:
    return float(np.linalg.norm(f - A @ u) / np.linalg.norm(f))


def jacobi_pcg(A: sp.spmatrix, f: np.ndarray, u0=None, rtol=1e-8, max_iter=100000):
    """Jacobi-PCG to ||f - A u|| <= rtol ||f|| (recurrence residual).

    Returns (u, iterations, recurrence relative residual, seconds)."""
    A = A.tocsr()
    f = np.asarray(f, np.float64)
    dinv = 1.0 / A.diagonal()
    u = np.zeros_like(f) if u0 is None else np.array(u0, np.float64)
    t0 = time.perf_counter()
    r = f - A @ u
    fn = np.linalg.norm(f)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rn = np.linalg.norm(r)
    while rn > rtol * fn and it < max_iter:
        q = A @ p
        alpha = rz / (p @ q)
        u += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        rn = np.linalg.norm(r)
        it += 1
    return u, it, rn / fn, time.perf_counter() - t0


def pcg(A: sp.spmatrix, f: np.ndarray, prec, u0=None, rtol=1e-8, max_iter=100000):
    """PCG with the SPD preconditioner z = prec(r), to ||f - A u|| <= rtol ||f|| (recurrence
    residual).  Returns (u, iterations, recurrence relative residual)."""
    A = A.tocsr()
    f = np.asarray(f, np.float64)
    u = np.zeros_like(f) if u0 is None else np.array(u0, np.float64)
    r = f - A @ u
    fn = np.linalg.norm(f)
    z = prec(r)
    p = z.copy()
    rz = r @ z
    it = 0
    rn = np.linalg.norm(r)
    while rn > rtol * fn and it < max_iter:
        q = A @ p
        alpha = rz / (p @ q)
        u += alpha * p
        r -= alpha * q
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        rn = np.linalg.norm(r)
        it += 1
    return u, it, rn / fn


def grid_prolongation(mesh, g: int) -> sp.csr_matrix:
    """P (free DOFs x 3 cells): the trilinear prolongation of cell-centred values on the
    level-g grid (oracle.learn.prolong, linear extrapolation at the boundary) at the free
    nodes, per displacement component (DOF 3 node + c, coarse DOF 3 cell + c)."""
    from . import fem as F
    from . import learn as LR
    X, Y, Z = LR.grid_shape(mesh, g)
    ncell = X * Y * Z
    cols = []
    for c in range(ncell):
        e = np.zeros(ncell)
        e[c] = 1.0
        cols.append(sp.csr_matrix(LR.prolong(mesh, e.reshape(X, Y, Z, 1), g)[:, :1]))
    Pn = sp.hstack(cols).tocsr()                     # nodes x cells
    Pf = Pn[F.free_nodes(mesh)]
    return sp.kron(Pf, sp.eye(3)).tocsr()


def coarse_correction(A: sp.spmatrix, P: sp.spmatrix):
    """r -> P (P^T A P)^-1 P^T r (Galerkin coarse correction), by a sparse LU of P^T A P."""
    lu = spla.splu((P.T @ A @ P).tocsc())
    return lambda r: P @ lu.solve(P.T @ np.asarray(r, np.float64))


def twolevel_pcg(A: sp.spmatrix, f: np.ndarray, P: sp.spmatrix, u0=None, rtol=1e-8, max_iter=100000):
    """PCG with M^-1 r = D^-1 r + P (P^T A P)^-1 P^T r.  Returns (u, iterations, residual)."""
    dinv = 1.0 / A.diagonal()
    cc = coarse_correction(A, P)
    return pcg(A, f, lambda r: dinv * r + cc(r), u0, rtol, max_iter)


def cell_transfer(X: int, Y: int, Z: int) -> sp.csr_matrix:
    """(3 fine cells x 3 coarse cells): trilinear interpolation from the cell centres of the
    (X/2, Y/2, Z/2) grid to those of the (X, Y, Z) grid (X, Y, Z even), linear extrapolation in
    the boundary half-cells (exact for linear fields); DOF 3 cell + c."""
    Xc, Yc, Zc = X // 2, Y // 2, Z // 2

    def axis(nf, nc):
        t = (np.arange(nf) + 0.5) / 2 - 0.5          # fine centres in coarse-centre units
        if nc == 1:
            return np.zeros(nf, np.int64), np.zeros(nf)
        i0 = np.clip(np.floor(t).astype(np.int64), 0, nc - 2)
        return i0, t - i0

    ix, wx = axis(X, Xc)
    iy, wy = axis(Y, Yc)
    iz, wz = axis(Z, Zc)
    fine = np.arange(X * Y * Z).reshape(X, Y, Z)
    rows, cols, vals = [], [], []
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = ((wx if a else 1 - wx)[:, None, None] * (wy if b else 1 - wy)[None, :, None]
                     * (wz if c else 1 - wz)[None, None, :])
                cx = np.minimum(ix + a, Xc - 1)[:, None, None]
                cy = np.minimum(iy + b, Yc - 1)[None, :, None]
                cz = np.minimum(iz + c, Zc - 1)[None, None, :]
                rows.append(fine.ravel())
                cols.append(np.broadcast_to((cx * Yc + cy) * Zc + cz, (X, Y, Z)).ravel())
                vals.append(np.broadcast_to(w, (X, Y, Z)).ravel())
    T = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(X * Y * Z, Xc * Yc * Zc))
    T.sum_duplicates()
    return sp.kron(T, sp.eye(3)).tocsr()


class VCycle:
    """V(nu, nu) cycle for a Galerkin operator Ac on the cell grid `shape` (3 DOFs per cell)."""

    def __init__(self, Ac: sp.spmatrix, shape, nu: int = 2, coarsest_cells: int = 64, power_steps: int = 50):
        self.nu = nu
        self.levels = []
        X, Y, Z = shape
        A = Ac.tocsr()
        while True:
            dinv = 1.0 / A.diagonal()
            v = np.random.default_rng(0).standard_normal(A.shape[0])
            lam = 1.0
            for _ in range(power_steps):             # lambda_max(D^-1 A) by power iteration
                v = dinv * (A @ v)
                lam = np.linalg.norm(v)
                v /= lam
            lev = {"A": A, "dinv": dinv, "omega": 1.0 / lam}
            self.levels.append(lev)
            if X * Y * Z <= coarsest_cells or X % 2 or Y % 2 or Z % 2:
                lev["lu"] = spla.splu(A.tocsc())
                break
            T = cell_transfer(X, Y, Z)
            lev["T"] = T
            A = (T.T @ A @ T).tocsr()
            X, Y, Z = X // 2, Y // 2, Z // 2

    def apply(self, r, k: int = 0):
        lev = self.levels[k]
        if "lu" in lev:
            return lev["lu"].solve(r)
        A, dinv, w = lev["A"], lev["dinv"], lev["omega"]
        x = np.zeros_like(r)
        for _ in range(self.nu):
            x += w * dinv * (r - A @ x)
        x += lev["T"] @ self.apply(lev["T"].T @ (r - A @ x), k + 1)
        for _ in range(self.nu):
            x += w * dinv * (r - A @ x)
        return x


def twolevel_vcycle_pcg(A: sp.spmatrix, f: np.ndarray, P: sp.spmatrix, shape, nu: int = 2, u0=None, rtol=1e-8,
                        max_iter=100000):
    """PCG with M^-1 r = D^-1 r + P V(P^T r), V a V-cycle for P^T A P on the grid `shape`."""
    dinv = 1.0 / A.diagonal()
    V = VCycle((P.T @ A @ P).tocsr(), shape, nu)
    return pcg(A, f, lambda r: dinv * r + P @ V.apply(P.T @ r), u0, rtol, max_iter)
