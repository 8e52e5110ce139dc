"""Pin of the oracle's C/OpenMP Jacobi-PCG (oracle/pcg_omp.c, the timed CPU baseline): it reaches
the direct solution of the reduced system, and it takes the iterations of the Python Jacobi-PCG
(oracle.solve.jacobi_pcg, the same algorithm) within 2 % (the dot products sum in another order)."""
import numpy as np

import workloads as W
from oracle import cpcg
from oracle import fem as F
from oracle import mesh as M
from oracle import solve as S


def test_c_jacobi_pcg_reaches_the_direct_solution_like_the_python_one():
    w = W.config1b()
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
    A, f, _ = F.reduced_system(m, w.rho[m.perm], w.load_nodes, w.load_comp, w.load_val)
    u, it, rel, _ = cpcg.jacobi_pcg(A, f, rtol=1e-10)
    assert rel <= 1e-10
    assert np.linalg.norm(f - A @ u) <= 1.01e-10 * np.linalg.norm(f)
    ud = S.direct(A, f)
    e = u - ud
    assert np.sqrt(e @ (A @ e) / (ud @ (A @ ud))) <= 1e-7
    _, it_py, _, _ = S.jacobi_pcg(A, f, rtol=1e-10)
    assert abs(it - it_py) <= 0.02 * it_py
    # a warm start at the solution needs no iteration
    _, it0, _, _ = cpcg.jacobi_pcg(A, f, u0=ud, rtol=1e-8)
    assert it0 == 0
    assert cpcg.threads() >= 1
