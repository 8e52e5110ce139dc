"""GPU parity of the adaptation step (paper Sec. 4) and the design difference (Eq. 10)
against the oracle: marks and adapted meshes bit for bit, D to rounding."""
import numpy as np
import pytest

import workloads as W
from oracle import amr as A
from oracle import mesh as M
from tests.gpu_common import ctx, tm

pytestmark = pytest.mark.gpu


def _moved_design(m, h_min, seed, r0=0.09):
    phi = W.truss_sdf(m.centres, seed, r0=r0)
    return np.clip(0.5 - phi / (2.0 * h_min), 1e-3, 1.0)


def _upload(w):
    d = w.dom
    return tm().tm_mesh_upload(ctx(), d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, w.E0, w.Emin, w.nu,
                               w.penal)


@pytest.mark.parametrize("seed,r_cells,rho_s", [(1, 1.6, 0.5), (2, 1.3, 0.5), (4, 3.7, 0.3), (1, 0.0, 0.5),
                                               (2, 2.0, 0.5), (4, 1.0, 0.5), (1, 4.0, 0.5)])
def test_marks_and_adapted_mesh_bit_exact(seed, r_cells, rho_s):
    import torch
    w = W.config1b(seed)
    d = w.dom
    _upload(w)
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    rho = _moved_design(m, d.h_min, seed + 7)
    rho_d = torch.as_tensor(rho, device="cuda:0")
    mk = torch.empty(m.Ne, dtype=torch.int8, device="cuda:0")
    tm().tm_amr_mark(ctx(), rho_d, rho_s, r_cells * d.h_min, mk)
    got = mk.cpu().numpy()
    want = A.final_marks(m, rho, rho_s, r_cells * d.h_min)
    np.testing.assert_array_equal(got, want)
    gl, gr = tm().tm_amr_adapt(ctx(), mk, rho_d)
    wl, wr = A.adapt(m, want, rho)
    np.testing.assert_array_equal(gl, wl)
    assert gr.tobytes() == wr.tobytes()


def test_design_difference_matches_oracle():
    import torch
    w = W.config1b(2)
    d = w.dom
    _upload(w)
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    rho = _moved_design(m, d.h_min, 9)
    rho_d = torch.as_tensor(rho, device="cuda:0")
    # the same design: exactly zero
    assert tm().tm_design_difference(ctx(), rho_d, m.leaves, rho) == 0.0
    # another design on another mesh (the adapted one, with a perturbed density), leaves shuffled
    marks = A.final_marks(m, rho, 0.5, 1.6 * d.h_min)
    l2, r2 = A.adapt(m, marks, rho)
    r2 = np.clip(r2 + 0.05 * np.sin(np.arange(r2.size)), 1e-3, 1.0)
    perm = np.random.default_rng(3).permutation(r2.size)
    got = tm().tm_design_difference(ctx(), rho_d, l2[perm], r2[perm])
    want = A.design_difference(d.nx, d.ny, d.nz, d.L, m.leaves, rho, l2, r2)
    assert got == pytest.approx(want, rel=1e-12)
    # uniform other design: |a - b| / a summed over cells
    u = W.uniform_leaves(d)
    got = tm().tm_design_difference(ctx(), rho_d, u, np.full(len(u), 0.25))
    want = A.design_difference(d.nx, d.ny, d.nz, d.L, m.leaves, rho, u, np.full(len(u), 0.25))
    assert got == pytest.approx(want, rel=1e-12)


def test_amr_rejections():
    import torch
    w = W.config1b(1)
    d = w.dom
    info = _upload(w)
    rho_d = torch.full((info["Ne"],), 0.5, dtype=torch.float64, device="cuda:0")
    mk = torch.empty(info["Ne"], dtype=torch.int8, device="cuda:0")
    with pytest.raises(tm().TmError):
        tm().tm_amr_mark(ctx(), rho_d, 0.5, 4.5 * d.h_min, mk)
    u = W.uniform_leaves(d)
    with pytest.raises(tm().TmError):          # a gap: one base cell missing
        tm().tm_design_difference(ctx(), rho_d, u[1:], np.full(len(u) - 1, 0.5))
    with pytest.raises(tm().TmError):          # an overlap that keeps the total volume
        bad = u.copy()
        bad[1] = bad[0]
        tm().tm_design_difference(ctx(), rho_d, bad, np.full(len(u), 0.5))
    bad = np.zeros(info["Ne"], np.int8)
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    bad[np.nonzero(m.leaves[:, 3] == d.L)[0][0]] = 1
    with pytest.raises(tm().TmError):
        tm().tm_amr_adapt(ctx(), torch.as_tensor(bad, device="cuda:0"), rho_d)
