"""The FP32 operator on several vectors at once (tm_apply_K_f32_multi): each result equals
the single-vector operator bit for bit, and meets the operator parity bound against the
oracle's assembled C^T K C."""
import numpy as np
import pytest

from tests.gpu_common import U32, case, ctx, tm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nrhs", [("config1", 1), ("config1b", 3), ("config1b", 4), ("small_truss", 4)])
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
    X = torch.zeros((5, 3 * c.m.Nn), dtype=torch.float32, device=c.dev)
    with pytest.raises(P.TmError):
        P.tm_apply_K_f32_multi(ctx(), c.t(c.rho), X, torch.zeros_like(X))
