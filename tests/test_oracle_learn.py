"""Pins for the oracle of the learned initial guess (oracle/learn.py): the convolution
convention against a loop, pooling/upsampling adjointness, the U-Net's gradients against
finite differences, exact grid transfers, load homogeneity and the energy loss."""
import numpy as np
import pytest

import workloads as W
from oracle import amr as AMR
from oracle import fem as F
from oracle import learn as LR
from oracle import mesh as M
from oracle import solve as S

torch = pytest.importorskip("torch")


def test_conv3d_is_the_zero_padded_cross_correlation():
    import torch.nn.functional as TF
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 4, 3, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    got = TF.conv3d(torch.tensor(x), torch.tensor(w), torch.tensor(b), padding=1).numpy()
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    want = np.zeros((1, 3, 4, 3, 5))
    for o in range(3):
        for i in range(4):
            for j in range(3):
                for k in range(5):
                    want[0, o, i, j, k] = b[o] + np.sum(w[o] * xp[0, :, i:i + 3, j:j + 3, k:k + 3])
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_pooling_and_upsampling_are_adjoint_up_to_eight():
    import torch.nn.functional as TF
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.standard_normal((1, 2, 6, 4, 8)))
    y = torch.tensor(rng.standard_normal((1, 2, 3, 2, 4)))
    lhs = float((TF.avg_pool3d(x, 2) * y).sum())
    rhs = float((x * TF.interpolate(y, scale_factor=2, mode="nearest")).sum()) / 8
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_unet_parameter_count():
    shapes = LR.unet_shapes((32, 64, 128))
    n = sum(int(np.prod(s)) for _, s in shapes)
    conv = lambda ci, co: co * ci * 27 + co
    want = (conv(4, 32) + conv(32, 32) + conv(32, 64) + conv(64, 64) + conv(64, 128) + conv(128, 128)
            + conv(128 + 64, 64) + conv(64, 64) + conv(64 + 32, 32) + conv(32, 32) + (3 * 32 + 3))
    assert n == want and 1.0e6 < n < 2.5e6


def test_unet_gradients_against_finite_differences():
    shapes = LR.unet_shapes((2, 3), c_in=4)
    params = [torch.tensor(p, requires_grad=True) for p in W.unet_init(shapes, seed=3)]
    x = torch.tensor(np.random.default_rng(4).standard_normal((1, 4, 4, 4, 4)), requires_grad=True)
    fn = lambda x_, *ps: LR.unet_forward(list(ps), x_)
    assert torch.autograd.gradcheck(fn, (x, *params), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_unet_shapes_and_level_halving():
    shapes = LR.unet_shapes((4, 6, 8))
    params = [torch.tensor(p) for p in W.unet_init(shapes, seed=1)]
    x = torch.zeros((2, 4, 8, 4, 12), dtype=torch.float64)
    y = LR.unet_forward(params, x)
    assert tuple(y.shape) == (2, 3, 8, 4, 12)


@pytest.mark.parametrize("g", [0, 1, 2])
def test_voxel_density_conserves_the_integral_and_matches_block_averages(g):
    w = W.config1b(2)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    rho = w.rho[m.perm]
    vox = LR.voxel_density(m, rho, g)
    vs = 1 << (d.L - g)
    total = float(np.sum(rho * m.size.astype(np.float64) ** 3))
    assert float(vox.sum()) * vs ** 3 == pytest.approx(total, rel=1e-13)
    fine = AMR.rasterize(d.nx, d.ny, d.nz, d.L, m.leaves, rho)          # finest cells, independent path
    X, Y, Z = vox.shape
    blocks = fine.reshape(X, vs, Y, vs, Z, vs).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(vox, blocks, rtol=1e-13, atol=1e-15)


def test_prolongation_is_exact_for_linear_fields_and_restriction_is_its_transpose():
    w = W.config1b(1)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    X, Y, Z = LR.grid_shape(m, 1)
    hv = 1 << (d.L - 1)
    cx, cy, cz = np.meshgrid((np.arange(X) + 0.5) * hv, (np.arange(Y) + 0.5) * hv, (np.arange(Z) + 0.5) * hv,
                             indexing="ij")
    a = np.array([0.3, -1.2, 2.0])
    B = np.array([[0.5, -0.25, 1.0], [2.0, 0.75, -1.5], [-0.125, 0.3, 0.6]])
    cells = a + np.stack([cx, cy, cz], -1) @ B.T
    got = LR.prolong(m, cells, 1)
    want = a + m.nodes.astype(np.float64) @ B.T
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    rng = np.random.default_rng(7)
    c = rng.standard_normal((X, Y, Z, 3))
    n = rng.standard_normal((m.Nn, 3))
    assert float(np.sum(LR.prolong(m, c, 1) * n)) == pytest.approx(float(np.sum(c * LR.restrict(m, n, 1))),
                                                                  rel=1e-12)


def test_initial_guess_is_homogeneous_in_the_loads():
    w = W.config1b(1)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    rho = w.rho[m.perm]
    f_full = F.full_load(m, w.load_nodes, w.load_comp, w.load_val)
    shapes = LR.unet_shapes((2, 3))
    params = [torch.tensor(p) for p in W.unet_init(shapes, seed=5)]
    outs = []
    for k in (1.0, 2.0):
        x, s = LR.network_input(m, rho, k * f_full)
        out = LR.unet_forward(params, torch.tensor(x)[None])[0].numpy()
        outs.append(LR.initial_guess(m, out, s))
    assert np.array_equal(outs[1], 2.0 * outs[0])
    # constrained DOFs (hanging, Dirichlet) are zero in the A-space layout
    free = np.zeros(m.Nn, bool)
    free[F.free_nodes(m)] = True
    assert np.all(outs[0].reshape(-1, 3)[~free] == 0.0) and np.any(outs[0] != 0.0)


def test_energy_loss_is_the_energy_error_up_to_a_constant():
    w = W.config1b(1)
    d = w.dom
    m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves)
    A, f, C = F.reduced_system(m, w.rho[m.perm], w.load_nodes, w.load_comp, w.load_val)
    us = S.direct(A, f)
    rng = np.random.default_rng(8)
    u0 = us + 1e-3 * np.abs(us).max() * rng.standard_normal(us.size)
    e = u0 - us
    want = 0.5 * float(e @ (A @ e)) - 0.5 * float(f @ us)
    assert LR.energy_loss(A, f, u0) == pytest.approx(want, rel=1e-9)
    # gradient A u0 - f, by a central difference along a random direction
    v = rng.standard_normal(us.size)
    h = 1e-4 * np.abs(us).max()
    fd = (LR.energy_loss(A, f, u0 + h * v) - LR.energy_loss(A, f, u0 - h * v)) / (2 * h)
    assert fd == pytest.approx(float((A @ u0 - f) @ v), rel=1e-6)
