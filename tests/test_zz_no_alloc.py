"""The no-allocation FP32 operator (tm_apply_K_f32_static) against the regular one.

tm_apply_K_f32_static serves callers that cannot allocate device memory when they
call (a stream being captured into a CUDA graph, a fixed memory budget, hosts that
forbid cudaMalloc after start-up): its scratch sits in a static device array.  This
test calls it twice in a row through the C ABI, with different inputs, and compares
each result with tm_apply_K_f32 on the same input, within the operator tolerance of
the parity tests (256 u32 (|A| |x|)_i per entry).  It lives in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest

from tests.gpu_common import U32, case, ctx, tm

pytestmark = pytest.mark.gpu


def test_static_scratch_operator_matches_regular_operator_twice():
    import torch
    c = case("small_truss")
    c.upload()
    rho = c.t(c.rho)
    bound_abs = abs(c.A)
    for seed in (21, 22):
        rng = np.random.default_rng(seed)
        x = rng.standard_normal(c.A.shape[0]).astype(np.float32).astype(np.float64)
        xd = c.t(c.full(x), torch.float32)
        y_ref = torch.zeros_like(xd)
        y_st = torch.full_like(xd, 3.0)
        tm().tm_apply_K_f32(ctx(), rho, xd, y_ref)
        tm().tm_apply_K_f32_static(ctx(), rho, xd, y_st)
        torch.cuda.synchronize()
        a = y_st.double().cpu().numpy()
        b = y_ref.double().cpu().numpy()
        tol = 256 * U32 * c.full(bound_abs @ np.abs(x))
        assert np.all(np.abs(a - b) <= tol)
        # constrained DOFs are written as 0 like the regular entry point
        cons = np.ones(a.size, bool)
        cons.reshape(-1, 3)[c.fn] = False
        assert np.all(a[cons] == 0.0)
