"""Oracle linear solvers for the reduced system A u = f (paper Sec. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``direct`` -- sparse LU of A (SciPy SuperLU), the reference solution.
* ``dense_cholesky`` -- a textbook column Cholesky, written out, for tiny systems
  (an independent check on the sparse factorisation).
* ``twolevel_pcg`` -- PCG with the additive two-level preconditioner
  M^-1 = D^-1 + P (P^T A P)^-1 P^T (Jacobi plus a Galerkin coarse correction on a
  coarse space given by a prolongation P, e.g. ``grid_prolongation``); no paper
  counterpart: the coarse-grid correction of the learned part's extension.
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
