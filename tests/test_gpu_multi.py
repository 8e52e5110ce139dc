"""The FP32 operator on several vectors at once (tm_apply_K_f32_multi): each result equals
the single-vector operator bit for bit, and meets the operator parity bound against the
oracle's assembled C^T K C."""
import numpy as np
import pytest

from tests.gpu_common import U32, case, ctx, tm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nrhs", [("config1", 1), ("config1b", 3), ("config1b", 4), ("small_truss", 4),
                                       ("config1b", 8)])
def test_multi_vector_operator(name, nrhs):
    import torch
    P = tm()
    c = case(name)
    c.upload()
    n3 = 3 * c.m.Nn
    rng = np.random.default_rng(21)
    X = torch.as_tensor(rng.standard_normal((nrhs, n3)).astype(np.float32), device=c.dev)
    Y = torch.full_like(X, 7.0)
    rho = c.t(c.rho)
    P.tm_apply_K_f32_multi(ctx(), rho, X, Y)
    for r in range(nrhs):
        y1 = torch.zeros(n3, dtype=torch.float32, device=c.dev)
        P.tm_apply_K_f32(ctx(), rho, X[r].contiguous(), y1)
        torch.cuda.synchronize()
        a, b = Y[r].cpu().numpy(), y1.cpu().numpy()
        assert a.tobytes() == b.tobytes(), float(np.abs(a - b).max())
    # one of them against the oracle (free DOFs)
    x = c.free(X[nrhs - 1].double().cpu().numpy())
    err = np.abs(c.free(Y[nrhs - 1].double().cpu().numpy()) - c.A @ x)
    assert np.all(err <= 256 * U32 * (abs(c.A) @ np.abs(x)))


def test_multi_vector_operator_rejects_too_many_vectors():
    import torch
    P = tm()
    c = case("config1")
    c.upload()
    X = torch.zeros((9, 3 * c.m.Nn), dtype=torch.float32, device=c.dev)
    with pytest.raises(P.TmError):
        P.tm_apply_K_f32_multi(ctx(), c.t(c.rho), X, torch.zeros_like(X))


def _loads(c, k):
    """k load cases: point loads at the load node in each direction and combinations, then point
    loads at nodes on the tip face."""
    node = c.w.load_nodes
    loads = [(node, [2], [-1.0]), (node, [1], [-1.0]), (np.concatenate([node, node]), [0, 2], [1.0, -0.5])]
    tip = c.m.nodes[c.m.nodes[:, 0] == c.m.nodes[:, 0].max()]
    rng = np.random.default_rng(17)
    while len(loads) < k:
        p = tip[rng.integers(len(tip))][None]
        loads.append((p, [int(rng.integers(3))], [float(rng.choice([-1.0, 1.0]))]))
    return loads[:k]


@pytest.mark.parametrize("precond,nrhs,graphs", [(0, 3, False), (0, 8, True), (1, 3, False), (1, 8, True)])
def test_multi_load_solve_matches_single_solves(precond, nrhs, graphs):
    """Load cases of one design solved in lockstep, with the Jacobi and the two-level
    preconditioner, plain launches or graph batches: every u and iteration count equals the
    single mixed solve of that case bit for bit, and meets the solve parity criterion."""
    import torch
    from oracle import fem as F
    P = tm()
    c = case("config1b")
    c.upload()
    n3 = 3 * c.m.Nn
    loads = _loads(c, nrhs)
    Fd = torch.zeros((len(loads), n3), dtype=torch.float64, device=c.dev)
    for r, (nd, comp, val) in enumerate(loads):
        f = torch.zeros(n3, dtype=torch.float64, device=c.dev)
        P.tm_build_rhs(ctx(), nd, comp, val, f)
        Fd[r] = f
    rho = c.t(c.rho)
    U = torch.zeros_like(Fd)
    stats = P.tm_pcg_solve_multi(ctx(), rho, Fd, U, rtol=1e-8, max_iter=200000, graphs=graphs, precond=precond,
                                 check_every=16)
    torch.cuda.synchronize()
    for r, (nd, comp, val) in enumerate(loads):
        u1 = torch.zeros(n3, dtype=torch.float64, device=c.dev)
        st1 = P.tm_pcg_solve(ctx(), rho, Fd[r].contiguous(), u1, rtol=1e-8, max_iter=200000,
                             precision=P.TM_PREC_MIXED, precond=precond, check_every=16)
        torch.cuda.synchronize()
        assert stats[r]["iterations"] == st1["iterations"]
        assert U[r].cpu().numpy().tobytes() == u1.cpu().numpy().tobytes()
        fr = F.reduced_system(c.m, c.rho, nd, comp, val)[1]
        ur = c.free(U[r].cpu().numpy())
        assert np.linalg.norm(fr - c.A @ ur) / np.linalg.norm(fr) <= 1e-8 * (1 + 1e-3)
