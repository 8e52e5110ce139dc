"""The no-allocation FP32 operator (tm_apply_K_f32_static) against the regular one.

tm_apply_K_f32_static serves callers that cannot allocate device memory when they
call: services whose device memory is a pool fixed at start-up, hosts whose
allocator forbids cudaMalloc after initialisation, and plug-ins that may only use
the buffers they are handed.  Its scratch sits in a static device array.  These tests
call it through the C ABI:

* twice in a row, with different inputs, comparing each result with tm_apply_K_f32
  on the same input.  Both launch the same kernels on the same FP32 coefficients with
  the same summation order, so the results must be bitwise equal;
* on a uniform mesh one element larger than the static array allows, which must be
  rejected with TM_EINVAL and a message naming the sizes, before any launch.

The file is collected last, so a run that stops at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from tests.gpu_common import case, ctx, tm

pytestmark = pytest.mark.gpu


def test_static_scratch_operator_matches_regular_operator_twice():
    import torch
    c = case("small_truss")
    c.upload()
    rho = c.t(c.rho)
    for seed in (21, 22):
        rng = np.random.default_rng(seed)
        x = rng.standard_normal(c.A.shape[0]).astype(np.float32).astype(np.float64)
        xd = c.t(c.full(x), torch.float32)
        y_ref = torch.zeros_like(xd)
        y_st = torch.full_like(xd, 3.0)
        tm().tm_apply_K_f32(ctx(), rho, xd, y_ref)
        tm().tm_apply_K_f32_static(ctx(), rho, xd, y_st)
        torch.cuda.synchronize()
        a = y_st.cpu().numpy()
        b = y_ref.cpu().numpy()
        assert np.array_equal(a, b)
        assert np.all(np.isfinite(a)) and np.abs(a).max() > 0
        # constrained DOFs are written as 0 like the regular entry point
        cons = np.ones(a.size, bool)
        cons.reshape(-1, 3)[c.fn] = False
        assert np.all(a[cons] == 0.0)


def test_static_scratch_rejects_a_mesh_over_its_limit():
    import torch
    P = tm()
    limit = 1 << 21                        # elements the static array holds
    nx, ny, nz = 129, 128, 127             # 2,097,024 elements: within the limit ...
    assert nx * ny * nz < limit
    nx = 130                               # ... 2,113,280: over it
    assert nx * ny * nz > limit
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    leaves = np.concatenate([g, np.zeros((len(g), 1), np.int64)], 1)
    big = P.tm_create(0, stream=torch.cuda.current_stream())
    try:
        info = P.tm_mesh_upload(big, nx, ny, nz, 0, 1.0, leaves, 1, 1.0, 1e-9, 0.3, 3.0)
        assert info["Ne"] == nx * ny * nz
        rho = torch.ones(info["Ne"], dtype=torch.float64, device="cuda")
        x = torch.ones(3 * info["Nn"], dtype=torch.float32, device="cuda")
        y = torch.full_like(x, 7.0)
        with pytest.raises(P.TmError) as err:
            P.tm_apply_K_f32_static(big, rho, x, y)
        assert err.value.code == P.TM_EINVAL
        assert str(nx * ny * nz) in str(err.value) and str(limit) in str(err.value)
        torch.cuda.synchronize()
        assert bool((y == 7.0).all())      # rejected before any launch: y untouched
    finally:
        P.tm_destroy(big)
