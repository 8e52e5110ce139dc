"""Learned initial guess for PCG: a 3D U-Net on the voxel grid maps (rho, P^T f / s) to a
displacement field whose prolongation s P(out) starts the solve.  Training minimises the
potential energy 0.5 u0^T A u0 - f^T u0 of the guess (the energy-norm error of the start up to
a constant), whose gradient in u0 is A u0 - f.

This module only sequences library calls (include/tm.h): the network's forward and backward
passes (tm_unet_*), the transfers (tm_learn_*), the operator (tm_apply_K) and the optimiser
(tm_adam_step) all run in the library's kernels; torch holds the device buffers.  The initial
parameters are an input (drawn by the caller).
"""
from __future__ import annotations

from . import tm as T


class LearnedGuess:
    """A U-Net of the given channel widths on the level-g voxel grid of one mesh (ctx's)."""

    def __init__(self, ctx, channels, params, g: int = 1):
        import torch
        self.ctx = ctx
        self.channels = tuple(int(c) for c in channels)
        self.g = int(g)
        nx, ny, nz, L = ctx.mesh_desc
        self.grid = (nx << g, ny << g, nz << g)
        self.params = params.detach().to(torch.float32).contiguous().clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        desc = T.unet_desc(self.channels, 1, self.grid)
        if T.tm_unet_param_count(desc) != self.params.numel():
            raise ValueError("parameter count does not match the network")

    def _buffers(self, n):
        import torch
        desc = T.unet_desc(self.channels, n, self.grid)
        dev = self.params.device
        ws = torch.zeros(T.tm_unet_workspace_floats(desc), dtype=torch.float32, device=dev)
        y = torch.zeros((n, 3) + self.grid, dtype=torch.float32, device=dev)
        return desc, ws, y

    def inputs(self, rho, f):
        """(x (4, X, Y, Z) device tensor, s) for one design."""
        import torch
        x = torch.zeros((4,) + self.grid, dtype=torch.float32, device=self.params.device)
        s = T.tm_learn_input(self.ctx, rho, f, self.g, x)
        return x, s

    def guess(self, x, s, u0):
        """u0 (A-space FP64) = s P(net(x)) for one input."""
        desc, ws, y = self._buffers(1)
        T.tm_unet_forward(self.ctx, desc, self.params, x.reshape((1, 4) + self.grid), y, ws)
        T.tm_learn_guess(self.ctx, y[0], s, self.g, u0)

    def train_step(self, batch, lr=1e-3):
        """One Adam step on a list of designs (rho, f, x, s): the energy losses summed."""
        import torch
        n = len(batch)
        desc, ws, y = self._buffers(n)
        x = torch.stack([b[2] for b in batch])
        T.tm_unet_forward(self.ctx, desc, self.params, x, y, ws)
        dy = torch.zeros_like(y)
        nn3 = 3 * self.ctx.info["Nn"]
        u0 = torch.zeros(nn3, dtype=torch.float64, device=self.params.device)
        au0 = torch.zeros_like(u0)
        for i, (rho, f, _, s) in enumerate(batch):
            T.tm_learn_guess(self.ctx, y[i], s, self.g, u0)
            T.tm_apply_K(self.ctx, rho, u0, au0)
            T.tm_learn_output_grad(self.ctx, au0, f, s, self.g, dy[i])
        grads = torch.zeros_like(self.params)
        T.tm_unet_backward(self.ctx, desc, self.params, x, dy, grads, None, ws)
        self.step_count += 1
        T.tm_adam_step(self.ctx, self.params, grads, self.m, self.v, self.step_count, lr)
