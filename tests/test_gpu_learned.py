"""The learned initial guess on the GPU (paper_1009_4975_gb300.learned, the tm_learn_* and
tm_adam_step entry points) against the oracle (oracle/learn.py), and what training gains.

* Transfers: the network input (voxel densities and the scaled load restriction) and the guess
  u0 = s P(out) match the oracle's network_input and initial_guess.  The input is FP32 of an
  FP64 gather (1 u32 of each channel's scale plus FP64 rounding); the guess is an FP64 gather of
  FP32 outputs (1e-13 of its scale).
* The energy gradient s P^T (A u0 - f) at the network output matches the oracle's chain rule
  (FP32 of an FP64 gather: 4 u32 of the scale).
* One Adam step matches the update formula written out here in FP64 (FP32 rounding).
* Training: designs from an optimisation run on the GPU (config 1b); the network, trained on
  the GPU for 600 steps on the first designs, starts the solve on held-out designs with a smaller
  energy-norm error than the untrained network and than the zero start (by at least 5 %); the
  report gives the PCG iterations from each start and from the previous design's solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem as F
from oracle import learn as LR
from tests.gpu_common import U32, case, ctx, tm

pytestmark = pytest.mark.gpu


def _setup(name="config1b", g=1):
    import torch
    c = case(name)
    c.upload()
    rho = c.t(c.rho)
    f = c.t(c.full(c.f))
    return c, rho, f


def test_network_input_and_guess_match_the_oracle():
    import torch
    P = tm()
    c, rho, f = _setup()
    g = 1
    X, Y, Z = LR.grid_shape(c.m, g)
    x = torch.zeros((4, X, Y, Z), dtype=torch.float32, device="cuda")
    s = P.tm_learn_input(ctx(), rho, f, g, x)
    xo, so = LR.network_input(c.m, c.rho, c.full(c.f), g)
    assert abs(s - so) <= 1e-12 * so
    xg = x.double().cpu().numpy()
    for ch in range(4):
        scale = np.abs(xo[ch]).max()
        assert np.abs(xg[ch] - xo[ch]).max() <= 2 * U32 * scale + 1e-15, ch
    rng = np.random.default_rng(3)
    out = rng.standard_normal((3, X, Y, Z)).astype(np.float32)
    od = torch.as_tensor(out, device="cuda")
    u0 = torch.full((3 * c.m.Nn,), 5.0, dtype=torch.float64, device="cuda")
    P.tm_learn_guess(ctx(), od, s, g, u0)
    want = LR.initial_guess(c.m, out.astype(np.float64), s, g)
    assert np.abs(u0.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()


def test_energy_gradient_at_the_network_output_matches_the_oracle():
    import torch
    P = tm()
    c, rho, f = _setup()
    g = 1
    X, Y, Z = LR.grid_shape(c.m, g)
    x = torch.zeros((4, X, Y, Z), dtype=torch.float32, device="cuda")
    s = P.tm_learn_input(ctx(), rho, f, g, x)
    out = np.random.default_rng(4).standard_normal((3, X, Y, Z)).astype(np.float32)
    u0 = torch.zeros(3 * c.m.Nn, dtype=torch.float64, device="cuda")
    P.tm_learn_guess(ctx(), torch.as_tensor(out, device="cuda"), s, g, u0)
    au0 = torch.zeros_like(u0)
    P.tm_apply_K(ctx(), rho, u0, au0)
    dout = torch.zeros((3, X, Y, Z), dtype=torch.float32, device="cuda")
    P.tm_learn_output_grad(ctx(), au0, f, s, g, dout)
    # oracle: d/d(out) of 0.5 u0^T A u0 - f^T u0 with u0 = s P(out) is s P^T (A u0 - f)
    u0o = LR.initial_guess(c.m, out.astype(np.float64), s, g)
    res = c.full(c.A @ c.free(u0o) - c.f)
    want = s * np.moveaxis(LR.restrict(c.m, res.reshape(-1, 3), g), -1, 0)
    got = dout.double().cpu().numpy()
    assert np.abs(got - want).max() <= 4 * U32 * np.abs(want).max()


def test_adam_step_matches_the_update_formula():
    import torch
    P = tm()
    rng = np.random.default_rng(5)
    n = 1000
    p0 = rng.standard_normal(n).astype(np.float32)
    g1, g2 = (rng.standard_normal(n).astype(np.float32) for _ in range(2))
    p = torch.as_tensor(p0.copy(), device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    pe, me, ve = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t, gr in ((1, g1), (2, g2)):
        P.tm_adam_step(ctx(), p, torch.as_tensor(gr, device="cuda"), m, v, t, lr, b1, b2, eps)
        me = b1 * me + (1 - b1) * gr
        ve = b2 * ve + (1 - b2) * gr.astype(np.float64) ** 2
        pe = pe - lr * (me / (1 - b1 ** t)) / (np.sqrt(ve / (1 - b2 ** t)) + eps)
    assert np.abs(p.cpu().numpy() - pe).max() <= 64 * U32 * (np.abs(pe).max() + lr)


def _energy_error(P, rho, f, u, ustar, au):
    """||u - u*||_A / ||u*||_A with the FP64 operator."""
    import torch
    e = u - ustar
    P.tm_apply_K(ctx(), rho, e, au)
    num = float(torch.dot(e, au))
    P.tm_apply_K(ctx(), rho, ustar, au)
    return abs(num) ** 0.5 / float(torch.dot(ustar, au)) ** 0.5


def test_training_on_the_gpu_improves_the_initial_guess():
    import torch
    from paper_1009_4975_gb300.learned import LearnedGuess
    P = tm()
    c, rho, f = _setup()
    w = c.w
    # designs along an optimisation run (mixed two-level solves, warm starts)
    designs, sols = [], []
    u = torch.zeros_like(f)
    uf, dc, dch = torch.zeros_like(f), torch.zeros_like(rho), torch.zeros_like(rho)
    cur = rho.clone()
    for it in range(40):
        P.tm_pcg_solve(ctx(), cur, f, u, rtol=1e-10, max_iter=200000, precision=P.TM_PREC_MIXED,
                       precond=P.TM_PRECOND_TWOLEVEL)
        designs.append(cur.clone())
        sols.append(u.clone())
        P.tm_expand(ctx(), u, uf)
        P.tm_sensitivity(ctx(), cur, uf, dc)
        P.tm_filter(ctx(), cur, dc, w.r_min, 0, dch)
        new = torch.zeros_like(cur)
        P.tm_oc_update(ctx(), cur, dch, 0.3, 0.2, 0.5, w.rho_min, new)
        cur = new
    channels = (8, 16, 32)
    params = W.unet_init(LR.unet_shapes(channels), seed=7)
    flat = torch.tensor(np.concatenate([q.ravel() for q in params]), dtype=torch.float32, device="cuda")
    net = LearnedGuess(ctx(), channels, flat, g=1)
    untrained = LearnedGuess(ctx(), channels, flat, g=1)
    data = [(r, f) + net.inputs(r, f) for r in designs]
    train, held = data[:30], list(range(30, 40))
    rng = np.random.default_rng(8)
    for step in range(600):
        idx = rng.choice(len(train), size=4, replace=False)
        net.train_step([train[i] for i in idx], lr=3e-3)
    au = torch.zeros_like(f)
    u0 = torch.zeros_like(f)
    err_t, err_u, it_t, it_z, it_w = [], [], [], [], []
    for i in held:
        r, _, x, s = data[i]
        net.guess(x, s, u0)
        err_t.append(_energy_error(P, r, f, u0, sols[i], au))
        st = P.tm_pcg_solve(ctx(), r, f, u0.clone(), rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                            precond=P.TM_PRECOND_TWOLEVEL)
        it_t.append(st["iterations"])
        untrained.guess(x, s, u0)
        err_u.append(_energy_error(P, r, f, u0, sols[i], au))
        z = torch.zeros_like(f)
        it_z.append(P.tm_pcg_solve(ctx(), r, f, z, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                                   precond=P.TM_PRECOND_TWOLEVEL)["iterations"])
        wst = sols[i - 1].clone()
        it_w.append(P.tm_pcg_solve(ctx(), r, f, wst, rtol=1e-8, max_iter=200000, precision=P.TM_PREC_MIXED,
                                   precond=P.TM_PRECOND_TWOLEVEL)["iterations"])
    print("held-out energy error: trained %.3f, untrained %.3f (zero start 1.0)" % (np.mean(err_t), np.mean(err_u)))
    print("two-level PCG iterations to 1e-8: network %.1f, zero %.1f, previous design %.1f"
          % (np.mean(it_t), np.mean(it_z), np.mean(it_w)))
    assert np.mean(err_t) < 0.95 * min(1.0, np.mean(err_u))
