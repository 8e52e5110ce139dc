"""The U-Net's GPU forward and backward kernels against the oracle (oracle/learn.py, FP64
autograd): the output and the gradients of every parameter and of the input, for a small
network and for the full-width one (channels 32, 64, 128; 1.41M parameters).  FP32 sums of
at most a few thousand terms: relative agreement to 1e-4 of each tensor's largest value."""
import numpy as np
import pytest

import workloads as W
from oracle import learn as LR
from tests.gpu_common import ctx, tm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("channels,n,grid", [((4, 6, 8), 2, (8, 4, 4)), ((32, 64, 128), 1, (8, 8, 8)), ((5,), 1, (3, 2, 5))])
def test_unet_forward_and_gradients_match_the_oracle(channels, n, grid):
    import torch
    P = tm()
    shapes = LR.unet_shapes(channels)
    params = W.unet_init(shapes, seed=11)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((n, 4) + grid)
    dy = rng.standard_normal((n, 3) + grid)
    # oracle
    pt = [torch.tensor(p, requires_grad=True) for p in params]
    xt = torch.tensor(x, requires_grad=True)
    yt = LR.unet_forward(pt, xt)
    (yt * torch.tensor(dy)).sum().backward()
    # GPU
    desc = P.unet_desc(channels, n, grid)
    assert P.tm_unet_param_count(desc) == sum(p.size for p in params)
    dev = torch.device("cuda:0")
    flat = torch.tensor(np.concatenate([p.ravel() for p in params]), dtype=torch.float32, device=dev)
    xd = torch.tensor(x, dtype=torch.float32, device=dev)
    yd = torch.zeros((n, 3) + grid, dtype=torch.float32, device=dev)
    ws = torch.zeros(P.tm_unet_workspace_floats(desc), dtype=torch.float32, device=dev)
    P.tm_unet_forward(ctx(), desc, flat, xd, yd, ws)
    dyd = torch.tensor(dy, dtype=torch.float32, device=dev)
    dp = torch.zeros_like(flat)
    dx = torch.zeros_like(xd)
    P.tm_unet_backward(ctx(), desc, flat, xd, dyd, dp, dx, ws)
    torch.cuda.synchronize()

    def close(got, want):
        want = np.asarray(want)
        assert np.abs(np.asarray(got, np.float64) - want).max() <= 1e-4 * max(np.abs(want).max(), 1e-30)

    close(yd.cpu().numpy(), yt.detach().numpy())
    close(dx.cpu().numpy(), xt.grad.numpy())
    dph = dp.cpu().numpy()
    o = 0
    for (name, shape), t in zip(shapes, pt):
        k = int(np.prod(shape))
        close(dph[o:o + k].reshape(shape), t.grad.numpy())
        o += k


def test_unet_rejects_bad_descriptions():
    import torch
    P = tm()
    assert P.tm_unet_param_count(P.unet_desc((4, 6), 1, (5, 4, 4))) == -1      # 5 not a multiple of 2
    desc = P.unet_desc((4, 6), 1, (5, 4, 4))
    z = torch.zeros(8, dtype=torch.float32, device="cuda:0")
    with pytest.raises(P.TmError):
        P.tm_unet_forward(ctx(), desc, z, z, z, z)
