"""Oracle of the learned initial guess for PCG: grid transfers, the 3D U-Net and its loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper has no learned component; it is an extension of the method, and every choice
below is a reading made for it:

* **Grid.**  The uniform voxel grid of level ``g`` of the base mesh (default 1):
  ``(nx 2^g, ny 2^g, nz 2^g)`` cells of side ``hv = h0 / 2^g``, cell-centred values.
* **Density input.**  The volume average of rho over each voxel: a leaf finer than
  a voxel contributes its share, a coarser leaf covers several voxels with its own
  value.  The integral of rho is kept exactly.
* **Prolongation P** (cells -> mesh nodes).  Trilinear interpolation of the
  cell-centred values at each node's coordinates.  In the boundary half-cells it
  extrapolates linearly: the cell index is clamped to [0, n - 2] and the weight
  may leave [0, 1].  P is exact for fields linear in space.
* **Load input.**  The restriction P^T f of the nodal loads (the adjoint of P), per
  component, divided by s = max |P^T f| so that the network sees O(1) inputs.
* **Output.**  u0 = s * P(net(x)) at every node, then the A-space vector (free
  DOFs).  Scaling by the same s makes the prediction homogeneous of degree 1 in
  the loads, like the exact solution.
* **Network.**  A U-Net with levels of ``channels[i]`` features:
  - per level, two 3x3x3 convolutions (zero padding 1, bias) each followed by ReLU;
  - down: 2x2x2 average pooling; up: nearest-neighbour 2x upsampling, concatenation
    with the skip features, then the two convolutions of that level;
  - output: a 1x1x1 convolution to 3 channels (u_x, u_y, u_z).
* **Loss.**  The potential energy 0.5 u0^T A u0 - f^T u0 of the initial guess.  It
  equals 0.5 ||u0 - u*||_A^2 minus a constant, so minimising it minimises the
  energy-norm error with which PCG starts, and its gradient in u0 is A u0 - f (the
  negative initial residual); no reference solution is needed.

Convolution, pooling and upsampling are taken from PyTorch (CPU, FP64) as library
primitives; backward passes come from autograd.
"""
from __future__ import annotations

import numpy as np

from . import fem as F
from .mesh import Mesh


# ---------------------------------------------------------------- grid transfers
def grid_shape(mesh: Mesh, g: int = 1):
    return (mesh.nx << g, mesh.ny << g, mesh.nz << g)


def voxel_density(mesh: Mesh, rho, g: int = 1) -> np.ndarray:
    """(X, Y, Z) volume averages of rho over the level-g voxels."""
    if g > mesh.L:
        raise ValueError("voxel level above the mesh's finest level")
    rho = np.asarray(rho, np.float64)
    X, Y, Z = grid_shape(mesh, g)
    vs = 1 << (mesh.L - g)                        # voxel side in finest units
    acc = np.zeros((X, Y, Z))
    for e in range(mesh.Ne):
        ix, iy, iz, lvl = (int(v) for v in mesh.leaves[e])
        s = 1 << (mesh.L - lvl)
        if s >= vs:                               # covers whole voxels
            acc[ix // vs:(ix + s) // vs, iy // vs:(iy + s) // vs, iz // vs:(iz + s) // vs] += rho[e] * vs ** 3
        else:                                     # a share of one voxel
            acc[ix // vs, iy // vs, iz // vs] += rho[e] * s ** 3
    return acc / vs ** 3


def _axis_weights(coord, n, hv):
    """Cell index i0 (clamped to [0, n-2]) and weight w of cell i0 + 1 for positions `coord`."""
    t = coord / hv - 0.5
    i0 = np.clip(np.floor(t).astype(np.int64), 0, n - 2)
    return i0, t - i0


def prolong(mesh: Mesh, cells, g: int = 1) -> np.ndarray:
    """(Nn, C) trilinear interpolation of the cell-centred field `cells` (X, Y, Z, C) at the nodes."""
    cells = np.asarray(cells, np.float64)
    X, Y, Z = grid_shape(mesh, g)
    hv = float(1 << (mesh.L - g))                 # in finest units (node coordinates are integers)
    out = np.zeros((mesh.Nn, cells.shape[-1]))
    ix, wx = _axis_weights(mesh.nodes[:, 0], X, hv)
    iy, wy = _axis_weights(mesh.nodes[:, 1], Y, hv)
    iz, wz = _axis_weights(mesh.nodes[:, 2], Z, hv)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = (wx if a else 1 - wx) * (wy if b else 1 - wy) * (wz if c else 1 - wz)
                out += w[:, None] * cells[ix + a, iy + b, iz + c]
    return out


def restrict(mesh: Mesh, nodal, g: int = 1) -> np.ndarray:
    """P^T: (Nn, C) nodal values to (X, Y, Z, C) cells, the transpose of `prolong`."""
    nodal = np.asarray(nodal, np.float64)
    X, Y, Z = grid_shape(mesh, g)
    hv = float(1 << (mesh.L - g))
    out = np.zeros((X, Y, Z, nodal.shape[-1]))
    ix, wx = _axis_weights(mesh.nodes[:, 0], X, hv)
    iy, wy = _axis_weights(mesh.nodes[:, 1], Y, hv)
    iz, wz = _axis_weights(mesh.nodes[:, 2], Z, hv)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = (wx if a else 1 - wx) * (wy if b else 1 - wy) * (wz if c else 1 - wz)
                np.add.at(out, (ix + a, iy + b, iz + c), w[:, None] * nodal)
    return out


def network_input(mesh: Mesh, rho, f_full, g: int = 1):
    """(x (4, X, Y, Z), s): channels rho, (P^T f)_x, _y, _z / s with s = max |P^T f|."""
    pf = restrict(mesh, np.asarray(f_full).reshape(-1, 3), g)
    s = float(np.abs(pf).max())
    if s == 0.0:
        raise ValueError("zero load")
    x = np.concatenate([voxel_density(mesh, rho, g)[None], np.moveaxis(pf / s, -1, 0)], axis=0)
    return x, s


def initial_guess(mesh: Mesh, out_cells, s, g: int = 1) -> np.ndarray:
    """A-space vector (3 Nn, constrained entries 0) of u0 = s * P(out) from the network output (3, X, Y, Z)."""
    nodal = s * prolong(mesh, np.moveaxis(np.asarray(out_cells), 0, -1), g)
    return F.to_full_layout(mesh, F.from_full_layout(mesh, nodal.ravel()))


# ---------------------------------------------------------------- network
def unet_shapes(channels, c_in=4, c_out=3):
    """[(name, shape)] of the parameters, in the order unet_forward consumes them."""
    shapes = []
    prev = c_in
    for i, c in enumerate(channels):                        # encoder (last level: bottleneck)
        shapes += [(f"enc{i}.w1", (c, prev, 3, 3, 3)), (f"enc{i}.b1", (c,)),
                   (f"enc{i}.w2", (c, c, 3, 3, 3)), (f"enc{i}.b2", (c,))]
        prev = c
    for i in range(len(channels) - 2, -1, -1):              # decoder
        c = channels[i]
        shapes += [(f"dec{i}.w1", (c, prev + c, 3, 3, 3)), (f"dec{i}.b1", (c,)),
                   (f"dec{i}.w2", (c, c, 3, 3, 3)), (f"dec{i}.b2", (c,))]
        prev = c
    shapes += [("out.w", (c_out, prev, 1, 1, 1)), ("out.b", (c_out,))]
    return shapes


def unet_forward(params, x):
    """params: list of FP64 torch tensors in unet_shapes order; x: (N, 4, X, Y, Z) FP64 torch tensor.
    Each level halves X, Y, Z, which must be divisible by 2^(levels - 1)."""
    import torch
    import torch.nn.functional as TF
    it = iter(params)

    def conv2(h):
        w1, b1, w2, b2 = next(it), next(it), next(it), next(it)
        h = torch.relu(TF.conv3d(h, w1, b1, padding=1))
        return torch.relu(TF.conv3d(h, w2, b2, padding=1))

    n_levels = (len(params) - 2) // 8 + 1
    skips = []
    h = x
    for i in range(n_levels):
        h = conv2(h)
        if i < n_levels - 1:
            skips.append(h)
            h = TF.avg_pool3d(h, 2)
    for i in range(n_levels - 2, -1, -1):
        h = TF.interpolate(h, scale_factor=2, mode="nearest")
        h = conv2(torch.cat([h, skips[i]], dim=1))
    w, b = next(it), next(it)
    return TF.conv3d(h, w, b)


def energy_loss(A, f, u0_free):
    """0.5 u0^T A u0 - f^T u0 on the free DOFs (reduced system of fem.reduced_system)."""
    u0 = np.asarray(u0_free, np.float64)
    return 0.5 * float(u0 @ (A @ u0)) - float(f @ u0)
