"""ctypes binding of libtm (include/tm.h): argument marshalling only.

Every function has the name of its C entry point and forwards to it; device
arrays are torch CUDA tensors (their data pointers are passed through), host
arrays are numpy arrays.  There is no fallback: if libtm.so is missing or the
GPU is unusable the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtm.so")

TM_OK, TM_EINVAL, TM_ECUDA, TM_ENOTCONVERGED, TM_ENONFINITE, TM_ETIMEOUT, TM_ENOMEM, TM_ESTATE = range(8)
TM_PREC_FP64, TM_PREC_MIXED = 0, 1
TM_PRECOND_JACOBI, TM_PRECOND_TWOLEVEL = 0, 1
_NAMES = {1: "TM_EINVAL", 2: "TM_ECUDA", 3: "TM_ENOTCONVERGED", 4: "TM_ENONFINITE", 5: "TM_ETIMEOUT",
          6: "TM_ENOMEM", 7: "TM_ESTATE"}


class TmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class tm_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("max_level", C.c_int32),
                ("h0", C.c_double), ("n_leaves", C.c_int64), ("leaves", C.POINTER(C.c_int32)),
                ("dirichlet_faces", C.c_uint32), ("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double),
                ("penal", C.c_double)]


class tm_mesh_info(C.Structure):
    _fields_ = [("Ne", C.c_int64), ("Nn", C.c_int64), ("n_hanging", C.c_int64), ("n_dirichlet", C.c_int64),
                ("n_free", C.c_int64), ("n_blocks", C.c_int32), ("max_local", C.c_int32),
                ("n_shared", C.c_int64), ("device_bytes", C.c_int64), ("max_block_bytes", C.c_int32),
                ("n_bricks", C.c_int32)]


class tm_solve_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("inner_rtol", C.c_double), ("check_every", C.c_int32), ("no_graphs", C.c_int32),
                ("precond", C.c_int32), ("smooth_sweeps", C.c_int32)]


class tm_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("sweeps", C.c_int32), ("rel_residual", C.c_double),
                ("seconds", C.c_double), ("fp64_applies", C.c_int32), ("fp32_applies", C.c_int32),
                ("coarse_levels", C.c_int32), ("pad_", C.c_int32), ("setup_seconds", C.c_double)]


class tm_unet_desc(C.Structure):
    _fields_ = [("levels", C.c_int32), ("channels", C.c_int32 * 6), ("c_in", C.c_int32), ("c_out", C.c_int32),
                ("n", C.c_int32), ("x", C.c_int32), ("y", C.c_int32), ("z", C.c_int32)]


class tm_profile_data(C.Structure):
    _fields_ = [("launches", C.c_int64), ("apply32_count", C.c_int64), ("apply64_count", C.c_int64),
                ("apply32_ms", C.c_double), ("apply64_ms", C.c_double)]


EXPORTS = ["tm_create", "tm_destroy", "tm_set_stream", "tm_last_error", "tm_mesh_upload", "tm_mesh_tables",
           "tm_tables_build", "tm_tables_copy", "tm_tables_free", "tm_build_rhs", "tm_apply_K", "tm_apply_K_f32", "tm_apply_K_f32_static", "tm_apply_K_f32_multi", "tm_jacobi_diag", "tm_pcg_solve", "tm_pcg_solve_batch", "tm_pcg_solve_multi", "tm_expand",
           "tm_sensitivity", "tm_filter", "tm_oc_update", "tm_amr_mark", "tm_amr_adapt", "tm_design_difference",
           "tm_tables_adapt", "tm_tables_operator", "tm_tables_bricks", "tm_tables_diag", "tm_tables_transfer", "tm_unet_param_count", "tm_unet_workspace_floats",
           "tm_unet_forward", "tm_unet_backward", "tm_profile", "tm_profile_read", "tm_coarse_setup",
           "tm_coarse_cells", "tm_coarse_apply", "tm_coarse_restrict", "tm_coarse_prolong", "tm_coarse_vcycle", "tm_transfer_displacement", "tm_learn_input",
           "tm_learn_guess", "tm_learn_output_grad", "tm_adam_step"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtm.so (built by paper_1009_4975_gb300.build).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtm.so not built ({path}); run paper_1009_4975_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "tm_create": [C.POINTER(vp), C.c_int, vp],
        "tm_destroy": [vp],
        "tm_set_stream": [vp, vp],
        "tm_mesh_upload": [vp, C.POINTER(tm_mesh_desc), C.POINTER(tm_mesh_info)],
        "tm_mesh_tables": [vp, vp, vp, vp, vp, vp, vp],
        "tm_build_rhs": [vp, i64, vp, vp, vp, vp],
        "tm_apply_K": [vp, vp, vp, vp],
        "tm_apply_K_f32": [vp, vp, vp, vp],
        "tm_apply_K_f32_static": [vp, vp, vp, vp],
        "tm_apply_K_f32_multi": [vp, C.c_int, vp, vp, vp],
        "tm_jacobi_diag": [vp, vp, vp],
        "tm_pcg_solve": [vp, vp, vp, vp, C.POINTER(tm_solve_opts), C.POINTER(tm_solve_stats)],
        "tm_pcg_solve_batch": [C.c_int, vp, vp, vp, vp, C.POINTER(tm_solve_opts), vp, vp],
        "tm_pcg_solve_multi": [vp, C.c_int, vp, vp, vp, C.POINTER(tm_solve_opts), vp],
        "tm_expand": [vp, vp, vp],
        "tm_sensitivity": [vp, vp, vp, vp, C.POINTER(dbl)],
        "tm_filter": [vp, vp, vp, dbl, C.c_int, vp],
        "tm_oc_update": [vp, vp, vp, dbl, dbl, dbl, dbl, vp, C.POINTER(dbl)],
        "tm_amr_mark": [vp, vp, dbl, dbl, vp],
        "tm_amr_adapt": [vp, vp, vp, i64, vp, vp, C.POINTER(i64)],
        "tm_design_difference": [vp, vp, i64, vp, vp, C.POINTER(dbl)],
        "tm_tables_adapt": [vp, vp, vp, i64, vp, vp, C.POINTER(i64)],
        "tm_tables_operator": [vp, vp, vp, vp, vp, vp, C.POINTER(i64)],
        "tm_tables_bricks": [vp, vp, vp, vp, vp, vp],
        "tm_tables_diag": [vp, vp, vp, vp, vp, C.POINTER(i64), C.POINTER(i64)],
        "tm_tables_transfer": [vp, vp, i64, vp, vp],
        "tm_unet_forward": [vp, C.POINTER(tm_unet_desc), vp, vp, vp, vp],
        "tm_unet_backward": [vp, C.POINTER(tm_unet_desc), vp, vp, vp, vp, vp, vp],
        "tm_profile": [vp, C.c_int],
        "tm_coarse_setup": [vp, vp, vp, vp],
        "tm_coarse_cells": [vp, C.c_int, vp],
        "tm_coarse_apply": [vp, C.c_int, vp, vp],
        "tm_coarse_restrict": [vp, vp, vp],
        "tm_coarse_prolong": [vp, vp, vp],
        "tm_coarse_vcycle": [vp, vp, vp, C.c_int],
        "tm_transfer_displacement": [vp, vp, i64, vp, vp],
        "tm_learn_input": [vp, vp, vp, C.c_int, vp, C.POINTER(dbl)],
        "tm_learn_guess": [vp, vp, dbl, C.c_int, vp],
        "tm_learn_output_grad": [vp, vp, vp, dbl, C.c_int, vp],
        "tm_adam_step": [vp, i64, vp, vp, vp, vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float],
        "tm_profile_read": [vp, C.POINTER(tm_profile_data)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.tm_tables_build.argtypes = [C.POINTER(tm_mesh_desc), C.POINTER(vp), C.POINTER(tm_mesh_info), C.c_char_p,
                                    C.c_int]
    lib.tm_tables_build.restype = C.c_int
    lib.tm_tables_copy.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.tm_tables_copy.restype = C.c_int
    lib.tm_tables_free.argtypes = [vp]
    lib.tm_tables_free.restype = None
    for name in ("tm_unet_param_count", "tm_unet_workspace_floats"):
        fn = getattr(lib, name)
        fn.argtypes = [C.POINTER(tm_unet_desc)]
        fn.restype = C.c_int64
    lib.tm_last_error.argtypes = [vp]
    lib.tm_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor, with dtype and size checks."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Ctx:
    """A library context bound to one device and stream; holds at most one mesh."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device
        self.info = None
        self.coarse = None
        self.mesh_desc = None

    def check(self, rc):
        if rc != TM_OK:
            raise TmError(rc, load_library().tm_last_error(self.handle).decode())

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tm_destroy(self.handle)
            self.handle = None


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def tm_create(device: int = 0, stream=None) -> Ctx:
    lib = load_library()
    h = C.c_void_p()
    rc = lib.tm_create(C.byref(h), device, _stream_ptr(stream))
    if rc != TM_OK:
        raise TmError(rc, f"tm_create failed on device {device}")
    return Ctx(h, device)


def tm_destroy(ctx: Ctx):
    if ctx.handle:
        load_library().tm_destroy(ctx.handle)
        ctx.handle = None


def tm_set_stream(ctx: Ctx, stream=None):
    ctx.check(load_library().tm_set_stream(ctx.handle, _stream_ptr(stream)))


def tm_last_error(ctx: Ctx) -> str:
    return load_library().tm_last_error(ctx.handle).decode()


def tm_mesh_upload(ctx: Ctx, nx, ny, nz, max_level, h0, leaves, dirichlet_faces=1, E0=1.0, Emin=1e-9, nu=0.3,
                   penal=3.0) -> dict:
    lv = np.ascontiguousarray(np.asarray(leaves, np.int32).reshape(-1, 4))
    d = tm_mesh_desc(nx, ny, nz, max_level, h0, lv.shape[0], lv.ctypes.data_as(C.POINTER(C.c_int32)),
                     dirichlet_faces, E0, Emin, nu, penal)
    info = tm_mesh_info()
    ctx.check(load_library().tm_mesh_upload(ctx.handle, C.byref(d), C.byref(info)))
    ctx.info = {k: getattr(info, k) for k, _ in tm_mesh_info._fields_}
    ctx.mesh_desc = (int(nx), int(ny), int(nz), int(max_level))
    ctx.coarse = None
    return ctx.info


def _table_arrays(i):
    Ne, Nn, nh = i["Ne"], i["Nn"], i["n_hanging"]
    return {"perm": np.empty(Ne, np.int64), "node_xyz": np.empty((Nn, 3), np.int32),
            "conn": np.empty((Ne, 8), np.int32), "hang_node": np.empty(nh, np.int32),
            "hang_master": np.empty((nh, 4), np.int32), "node_flags": np.empty(Nn, np.uint8)}


def tm_mesh_tables(ctx: Ctx) -> dict:
    out = _table_arrays(ctx.info)
    ctx.check(load_library().tm_mesh_tables(ctx.handle, *[C.c_void_p(a.ctypes.data) for a in out.values()]))
    return out


def tm_tables_build(nx, ny, nz, max_level, h0, leaves, dirichlet_faces=1, E0=1.0, Emin=1e-9, nu=0.3,
                    penal=3.0):
    """Host-only table construction; returns (info, tables) or raises TmError(TM_EINVAL)."""
    lib = load_library()
    lv = np.ascontiguousarray(np.asarray(leaves, np.int32).reshape(-1, 4))
    d = tm_mesh_desc(nx, ny, nz, max_level, h0, lv.shape[0], lv.ctypes.data_as(C.POINTER(C.c_int32)),
                     dirichlet_faces, E0, Emin, nu, penal)
    info = tm_mesh_info()
    h = C.c_void_p()
    err = C.create_string_buffer(512)
    rc = lib.tm_tables_build(C.byref(d), C.byref(h), C.byref(info), err, 512)
    if rc != TM_OK:
        raise TmError(rc, err.value.decode())
    try:
        i = {k: getattr(info, k) for k, _ in tm_mesh_info._fields_}
        out = _table_arrays(i)
        rc = lib.tm_tables_copy(h, *[C.c_void_p(a.ctypes.data) for a in out.values()])
        if rc != TM_OK:
            raise TmError(rc, "tm_tables_copy failed")
        return i, out
    finally:
        lib.tm_tables_free(h)


def tm_build_rhs(ctx: Ctx, node_xyz, comp, val, f):
    nx = np.ascontiguousarray(np.asarray(node_xyz, np.int32).reshape(-1, 3))
    cp = np.ascontiguousarray(np.asarray(comp, np.int32).ravel())
    vl = np.ascontiguousarray(np.asarray(val, np.float64).ravel())
    import torch
    ctx.check(load_library().tm_build_rhs(ctx.handle, nx.shape[0], C.c_void_p(nx.ctypes.data),
                                          C.c_void_p(cp.ctypes.data), C.c_void_p(vl.ctypes.data),
                                          _ptr(f, torch.float64, 3 * ctx.info["Nn"], "f")))


def _vec(ctx, t, dtype, name):
    return _ptr(t, dtype, 3 * ctx.info["Nn"], name)


def _elem(ctx, t, name):
    import torch
    return _ptr(t, torch.float64, ctx.info["Ne"], name)


def tm_apply_K(ctx: Ctx, rho, x, y):
    import torch
    ctx.check(load_library().tm_apply_K(ctx.handle, _elem(ctx, rho, "rho"), _vec(ctx, x, torch.float64, "x"),
                                        _vec(ctx, y, torch.float64, "y")))


def tm_apply_K_f32(ctx: Ctx, rho, x, y):
    import torch
    ctx.check(load_library().tm_apply_K_f32(ctx.handle, _elem(ctx, rho, "rho"), _vec(ctx, x, torch.float32, "x"),
                                            _vec(ctx, y, torch.float32, "y")))


def tm_apply_K_f32_static(ctx: Ctx, rho, x, y):
    """FP32 operator that allocates nothing (scratch in a static device array); see include/tm.h."""
    import torch
    ctx.check(load_library().tm_apply_K_f32_static(ctx.handle, _elem(ctx, rho, "rho"),
                                                   _vec(ctx, x, torch.float32, "x"),
                                                   _vec(ctx, y, torch.float32, "y")))


def tm_apply_K_f32_multi(ctx: Ctx, rho, x, y):
    """FP32 operator on the rows of x (nrhs, 3 Nn) at once; see include/tm.h."""
    import torch
    if x.dim() != 2 or x.shape != y.shape or x.shape[1] != 3 * ctx.info["Nn"]:
        raise ValueError("x and y must be (nrhs, 3 Nn)")
    ctx.check(load_library().tm_apply_K_f32_multi(ctx.handle, x.shape[0], _elem(ctx, rho, "rho"),
                                                  _ptr(x, torch.float32, None, "x"), _ptr(y, torch.float32, None, "y")))


def tm_jacobi_diag(ctx: Ctx, rho, d):
    import torch
    ctx.check(load_library().tm_jacobi_diag(ctx.handle, _elem(ctx, rho, "rho"), _vec(ctx, d, torch.float64, "d")))


def tm_pcg_solve(ctx: Ctx, rho, f, u, rtol=1e-8, max_iter=100000, precision=TM_PREC_FP64, inner_rtol=0.1,
                 check_every=64, raise_on_error=True, graphs=True, precond=TM_PRECOND_JACOBI,
                 smooth_sweeps=1) -> dict:
    import torch
    o = tm_solve_opts(rtol, max_iter, precision, inner_rtol, check_every, 0 if graphs else 1, precond, smooth_sweeps)
    s = tm_solve_stats()
    rc = load_library().tm_pcg_solve(ctx.handle, _elem(ctx, rho, "rho"), _vec(ctx, f, torch.float64, "f"),
                                     _vec(ctx, u, torch.float64, "u"), C.byref(o), C.byref(s))
    stats = {k: getattr(s, k) for k, _ in tm_solve_stats._fields_}
    stats["status"] = rc
    if raise_on_error and rc != TM_OK:
        ctx.check(rc)
    return stats


def tm_pcg_solve_batch(ctxs, rhos, fs, us, rtol=1e-8, max_iter=100000, precision=TM_PREC_FP64, inner_rtol=0.1,
                       check_every=64, raise_on_error=True, graphs=True, precond=TM_PRECOND_JACOBI,
                       smooth_sweeps=1) -> list:
    """Independent solves on distinct contexts, run concurrently (include/tm.h)."""
    import torch
    n = len(ctxs)
    if not (len(rhos) == len(fs) == len(us) == n) or n == 0:
        raise ValueError("one rho, f and u per context")
    hs = (C.c_void_p * n)(*[c.handle for c in ctxs])
    rp = (C.c_void_p * n)(*[_elem(c, r, "rho").value for c, r in zip(ctxs, rhos)])
    fp = (C.c_void_p * n)(*[_vec(c, f, torch.float64, "f").value for c, f in zip(ctxs, fs)])
    up = (C.c_void_p * n)(*[_vec(c, u, torch.float64, "u").value for c, u in zip(ctxs, us)])
    o = tm_solve_opts(rtol, max_iter, precision, inner_rtol, check_every, 0 if graphs else 1, precond, smooth_sweeps)
    st = (tm_solve_stats * n)()
    status = (C.c_int * n)()
    rc = load_library().tm_pcg_solve_batch(n, hs, rp, fp, up, C.byref(o), st, status)
    out = []
    for i in range(n):
        d = {k: getattr(st[i], k) for k, _ in tm_solve_stats._fields_}
        d["status"] = status[i]
        out.append(d)
    if raise_on_error and rc != TM_OK:
        bad = next((i for i in range(n) if status[i] != TM_OK), 0)
        ctxs[bad].check(status[bad] if status[bad] != TM_OK else rc)
    return out


def tm_pcg_solve_multi(ctx: Ctx, rho, F, U, rtol=1e-8, max_iter=100000, inner_rtol=0.1, check_every=64,
                       raise_on_error=True, graphs=True, precond=TM_PRECOND_JACOBI, smooth_sweeps=1) -> list:
    """Mixed solves of the load cases in the rows of F (nrhs, 3 Nn) into U, in lockstep; see include/tm.h."""
    import torch
    if F.dim() != 2 or F.shape != U.shape or F.shape[1] != 3 * ctx.info["Nn"]:
        raise ValueError("F and U must be (nrhs, 3 Nn)")
    nr = F.shape[0]
    o = tm_solve_opts(rtol, max_iter, TM_PREC_MIXED, inner_rtol, check_every, 0 if graphs else 1, precond,
                      smooth_sweeps)
    st = (tm_solve_stats * nr)()
    rc = load_library().tm_pcg_solve_multi(ctx.handle, nr, _elem(ctx, rho, "rho"), _ptr(F, torch.float64, None, "F"),
                                           _ptr(U, torch.float64, None, "U"), C.byref(o), st)
    out = []
    for i in range(nr):
        d = {k: getattr(st[i], k) for k, _ in tm_solve_stats._fields_}
        d["status"] = rc
        out.append(d)
    if raise_on_error and rc != TM_OK:
        ctx.check(rc)
    return out


def tm_expand(ctx: Ctx, u, u_full):
    import torch
    ctx.check(load_library().tm_expand(ctx.handle, _vec(ctx, u, torch.float64, "u"),
                                       _vec(ctx, u_full, torch.float64, "u_full")))


def tm_sensitivity(ctx: Ctx, rho, u_full, dc) -> float:
    import torch
    c = C.c_double()
    ctx.check(load_library().tm_sensitivity(ctx.handle, _elem(ctx, rho, "rho"),
                                            _vec(ctx, u_full, torch.float64, "u_full"), _elem(ctx, dc, "dc"),
                                            C.byref(c)))
    return c.value


def tm_filter(ctx: Ctx, rho, x, rmin, mode, out):
    ctx.check(load_library().tm_filter(ctx.handle, _elem(ctx, rho, "rho"), _elem(ctx, x, "x"), rmin, mode,
                                       _elem(ctx, out, "out")))


def tm_oc_update(ctx: Ctx, rho, dc, volfrac, move, eta, rho_min, rho_new) -> float:
    ch = C.c_double()
    ctx.check(load_library().tm_oc_update(ctx.handle, _elem(ctx, rho, "rho"), _elem(ctx, dc, "dc"), volfrac, move,
                                          eta, rho_min, _elem(ctx, rho_new, "rho_new"), C.byref(ch)))
    return ch.value


def tm_amr_mark(ctx: Ctx, rho, rho_solid: float, r_amr: float, mark):
    """Adaptation marks (+1 / 0 / -1, int8 CUDA tensor of Ne) after both sweeps; see include/tm.h."""
    import torch
    ctx.check(load_library().tm_amr_mark(ctx.handle, _elem(ctx, rho, "rho"), rho_solid, r_amr,
                                         _ptr(mark, torch.int8, ctx.info["Ne"], "mark")))


def _adapt_call(fn, ne, handle, mark_p, rho_p, raise_err):
    cap = 8 * ne + 64
    for _ in range(2):
        lv = np.empty((cap, 4), np.int32)
        r = np.empty(cap, np.float64)
        n = C.c_int64(0)
        rc = fn(handle, mark_p, rho_p, cap, C.c_void_p(lv.ctypes.data), C.c_void_p(r.ctypes.data), C.byref(n))
        if rc == TM_OK:
            return lv[:n.value].copy(), r[:n.value].copy()
        if n.value <= cap:
            raise_err(rc)
        cap = n.value
    raise_err(rc)


def tm_amr_adapt(ctx: Ctx, mark, rho):
    """(leaves int32 (n, 4), rho float64 (n,)) of the adapted mesh, on the host."""
    import torch
    ne = ctx.info["Ne"]
    return _adapt_call(load_library().tm_amr_adapt, ne, ctx.handle, _ptr(mark, torch.int8, ne, "mark"),
                       _elem(ctx, rho, "rho"), ctx.check)


def tm_design_difference(ctx: Ctx, rho, leaves_other, rho_other) -> float:
    """Eq. 10 between the uploaded design and another one given on the host."""
    lv = np.ascontiguousarray(np.asarray(leaves_other, np.int32).reshape(-1, 4))
    ro = np.ascontiguousarray(np.asarray(rho_other, np.float64).ravel())
    if ro.size != lv.shape[0]:
        raise ValueError("rho_other must have one value per leaf")
    d = C.c_double()
    ctx.check(load_library().tm_design_difference(ctx.handle, _elem(ctx, rho, "rho"), lv.shape[0],
                                                  C.c_void_p(lv.ctypes.data), C.c_void_p(ro.ctypes.data),
                                                  C.byref(d)))
    return d.value


def tm_tables_adapt(nx, ny, nz, max_level, h0, leaves, mark, rho):
    """Host-only adaptation (tm_tables_adapt): marks and rho in the tables' (Morton) element order."""
    lib = load_library()
    lv = np.ascontiguousarray(np.asarray(leaves, np.int32).reshape(-1, 4))
    d = tm_mesh_desc(nx, ny, nz, max_level, h0, lv.shape[0], lv.ctypes.data_as(C.POINTER(C.c_int32)), 1, 1.0,
                     1e-9, 0.3, 3.0)
    info = tm_mesh_info()
    h = C.c_void_p()
    err = C.create_string_buffer(512)
    rc = lib.tm_tables_build(C.byref(d), C.byref(h), C.byref(info), err, 512)
    if rc != TM_OK:
        raise TmError(rc, err.value.decode())
    try:
        mk = np.ascontiguousarray(np.asarray(mark, np.int8).ravel())
        r = np.ascontiguousarray(np.asarray(rho, np.float64).ravel())
        if mk.size != info.Ne or r.size != info.Ne:
            raise ValueError("mark and rho must have Ne entries")

        def raise_err(code):
            raise TmError(code, "tm_tables_adapt rejected the marks")
        return _adapt_call(lib.tm_tables_adapt, info.Ne, h, C.c_void_p(mk.ctypes.data), C.c_void_p(r.ctypes.data),
                           raise_err)
    finally:
        lib.tm_tables_free(h)


def tm_tables_operator(nx, ny, nz, max_level, h0, leaves, dirichlet_faces=1):
    """Host-only export of the operator's block and brick tables (tm_tables_operator,
    tm_tables_bricks): dict with info, rec_off, brec (uint8), modal (8, 3, 3), sh_node, sh_ptr,
    brick_e0, brick_node, brick_hax, brick_out, brick_fold (bricks x 125)."""
    lib = load_library()
    lv = np.ascontiguousarray(np.asarray(leaves, np.int32).reshape(-1, 4))
    d = tm_mesh_desc(nx, ny, nz, max_level, h0, lv.shape[0], lv.ctypes.data_as(C.POINTER(C.c_int32)),
                     dirichlet_faces, 1.0, 1e-9, 0.3, 3.0)
    info = tm_mesh_info()
    h = C.c_void_p()
    err = C.create_string_buffer(512)
    rc = lib.tm_tables_build(C.byref(d), C.byref(h), C.byref(info), err, 512)
    if rc != TM_OK:
        raise TmError(rc, err.value.decode())
    try:
        nb = C.c_int64(0)
        lib.tm_tables_operator(h, None, None, None, None, None, C.byref(nb))
        out = {"info": {k: getattr(info, k) for k, _ in tm_mesh_info._fields_},
               "rec_off": np.zeros(info.n_blocks + 1, np.int32), "brec": np.zeros(nb.value, np.uint8),
               "modal": np.zeros((8, 3, 3)), "sh_node": np.zeros(info.n_shared, np.int32),
               "sh_ptr": np.zeros(info.n_shared + 1, np.int32)}
        rc = lib.tm_tables_operator(h, *[C.c_void_p(out[k].ctypes.data) for k in
                                         ("rec_off", "brec", "modal", "sh_node", "sh_ptr")], C.byref(nb))
        if rc != TM_OK:
            raise TmError(rc, "tm_tables_operator failed")
        nbk = info.n_bricks
        out.update(brick_e0=np.zeros(nbk, np.int32), brick_node=np.zeros((nbk, 125), np.int32),
                   brick_hax=np.zeros((nbk, 125), np.uint8), brick_out=np.zeros((nbk, 125), np.int32),
                   brick_fold=np.zeros((nbk, 125), np.uint32))
        rc = lib.tm_tables_bricks(h, *[C.c_void_p(out[k].ctypes.data) for k in
                                       ("brick_e0", "brick_node", "brick_hax", "brick_out", "brick_fold")])
        if rc != TM_OK:
            raise TmError(rc, "tm_tables_bricks failed")
        return out
    finally:
        lib.tm_tables_free(h)


def unet_desc(channels, n, grid, c_in=4, c_out=3) -> tm_unet_desc:
    ch = (C.c_int32 * 6)(*(list(channels) + [0] * (6 - len(channels))))
    return tm_unet_desc(len(channels), ch, c_in, c_out, n, *grid)


def tm_unet_param_count(desc: tm_unet_desc) -> int:
    return load_library().tm_unet_param_count(C.byref(desc))


def tm_unet_workspace_floats(desc: tm_unet_desc) -> int:
    return load_library().tm_unet_workspace_floats(C.byref(desc))


def tm_unet_forward(ctx: Ctx, desc: tm_unet_desc, params, x, y, ws):
    """y = net(x) (float32 CUDA tensors); see include/tm.h."""
    import torch
    ctx.check(load_library().tm_unet_forward(ctx.handle, C.byref(desc), _ptr(params, torch.float32, None, "params"),
                                             _ptr(x, torch.float32, None, "x"), _ptr(y, torch.float32, None, "y"),
                                             _ptr(ws, torch.float32, None, "ws")))


def tm_unet_backward(ctx: Ctx, desc: tm_unet_desc, params, x, dy, dparams, dx, ws):
    """dL/dparams (and dL/dx unless dx is None) from dy, after tm_unet_forward with the same ws."""
    import torch
    ctx.check(load_library().tm_unet_backward(ctx.handle, C.byref(desc), _ptr(params, torch.float32, None, "params"),
                                              _ptr(x, torch.float32, None, "x"), _ptr(dy, torch.float32, None, "dy"),
                                              _ptr(dparams, torch.float32, None, "dparams"),
                                              None if dx is None else _ptr(dx, torch.float32, None, "dx"),
                                              _ptr(ws, torch.float32, None, "ws")))


def tm_tables_diag(nx, ny, nz, max_level, h0, leaves, dirichlet_faces=1, nu=0.3):
    """Host-only export of the Jacobi-diagonal tables (tm_tables_diag): dict with info, ptr, elem,
    q (uint16), tab (triples x 3)."""
    lib = load_library()
    lv = np.ascontiguousarray(np.asarray(leaves, np.int32).reshape(-1, 4))
    d = tm_mesh_desc(nx, ny, nz, max_level, h0, lv.shape[0], lv.ctypes.data_as(C.POINTER(C.c_int32)),
                     dirichlet_faces, 1.0, 1e-9, nu, 3.0)
    info = tm_mesh_info()
    h = C.c_void_p()
    err = C.create_string_buffer(512)
    rc = lib.tm_tables_build(C.byref(d), C.byref(h), C.byref(info), err, 512)
    if rc != TM_OK:
        raise TmError(rc, err.value.decode())
    try:
        ne, nt = C.c_int64(0), C.c_int64(0)
        lib.tm_tables_diag(h, None, None, None, None, C.byref(ne), C.byref(nt))
        out = {"info": {k: getattr(info, k) for k, _ in tm_mesh_info._fields_},
               "ptr": np.zeros(info.Nn + 1, np.int32), "elem": np.zeros(ne.value, np.int32),
               "q": np.zeros(ne.value, np.uint16), "tab": np.zeros((nt.value, 3))}
        rc = lib.tm_tables_diag(h, *[C.c_void_p(out[k].ctypes.data) for k in ("ptr", "elem", "q", "tab")],
                                C.byref(ne), C.byref(nt))
        if rc != TM_OK:
            raise TmError(rc, "tm_tables_diag failed")
        return out
    finally:
        lib.tm_tables_free(h)


def tm_tables_transfer(nx, ny, nz, max_level, h0, leaves, u_full, points, dirichlet_faces=1):
    """Host-only: the field u_full (3 Nn, node order of the tables built from `leaves`) at the
    integer points (n, 3); returns (n, 3)."""
    lib = load_library()
    lv = np.ascontiguousarray(np.asarray(leaves, np.int32).reshape(-1, 4))
    d = tm_mesh_desc(nx, ny, nz, max_level, h0, lv.shape[0], lv.ctypes.data_as(C.POINTER(C.c_int32)),
                     dirichlet_faces, 1.0, 1e-9, 0.3, 3.0)
    info = tm_mesh_info()
    h = C.c_void_p()
    err = C.create_string_buffer(512)
    rc = lib.tm_tables_build(C.byref(d), C.byref(h), C.byref(info), err, 512)
    if rc != TM_OK:
        raise TmError(rc, err.value.decode())
    try:
        u = np.ascontiguousarray(np.asarray(u_full, np.float64).ravel())
        if u.size != 3 * info.Nn:
            raise ValueError("u_full must have 3 Nn entries")
        pts = np.ascontiguousarray(np.asarray(points, np.int32).reshape(-1, 3))
        out = np.zeros(pts.shape, np.float64)
        rc = lib.tm_tables_transfer(h, C.c_void_p(u.ctypes.data), pts.shape[0], C.c_void_p(pts.ctypes.data),
                                    C.c_void_p(out.ctypes.data))
        if rc != TM_OK:
            raise TmError(rc, "tm_tables_transfer: point outside the box")
        return out
    finally:
        lib.tm_tables_free(h)


def tm_profile(ctx: Ctx, enable: bool = True):
    ctx.check(load_library().tm_profile(ctx.handle, 1 if enable else 0))


def tm_profile_read(ctx: Ctx) -> dict:
    d = tm_profile_data()
    ctx.check(load_library().tm_profile_read(ctx.handle, C.byref(d)))
    return {k: getattr(d, k) for k, _ in tm_profile_data._fields_}


# ---------------------------------------------------------------- two-level preconditioner
def _lattice(ctx: Ctx, level: int) -> int:
    X, Y, Z = ctx.coarse["shapes"][level]
    return 3 * (X + 1) * (Y + 1) * (Z + 1)


def tm_coarse_setup(ctx: Ctx, rho) -> dict:
    """Level operators of the two-level preconditioner for rho; returns the levels' cell counts."""
    lv = C.c_int32(0)
    sh = (C.c_int32 * 36)()
    ctx.check(load_library().tm_coarse_setup(ctx.handle, _elem(ctx, rho, "rho"), C.byref(lv), sh))
    ctx.coarse = {"levels": lv.value, "shapes": [tuple(sh[3 * i:3 * i + 3]) for i in range(lv.value)]}
    return ctx.coarse


def tm_coarse_cells(ctx: Ctx, level: int, K):
    import torch
    X, Y, Z = ctx.coarse["shapes"][level]
    ctx.check(load_library().tm_coarse_cells(ctx.handle, level, _ptr(K, torch.float32, X * Y * Z * 576, "K")))


def tm_coarse_apply(ctx: Ctx, level: int, x, y):
    import torch
    n = _lattice(ctx, level)
    ctx.check(load_library().tm_coarse_apply(ctx.handle, level, _ptr(x, torch.float32, n, "x"),
                                             _ptr(y, torch.float32, n, "y")))


def tm_coarse_restrict(ctx: Ctx, r, b0):
    import torch
    ctx.check(load_library().tm_coarse_restrict(ctx.handle, _vec(ctx, r, torch.float32, "r"),
                                                _ptr(b0, torch.float32, _lattice(ctx, 0), "b0")))


def tm_coarse_prolong(ctx: Ctx, v0, y):
    import torch
    ctx.check(load_library().tm_coarse_prolong(ctx.handle, _ptr(v0, torch.float32, _lattice(ctx, 0), "v0"),
                                               _vec(ctx, y, torch.float32, "y")))


def tm_coarse_vcycle(ctx: Ctx, b0, x0, nu=1):
    import torch
    n = _lattice(ctx, 0)
    ctx.check(load_library().tm_coarse_vcycle(ctx.handle, _ptr(b0, torch.float32, n, "b0"),
                                              _ptr(x0, torch.float32, n, "x0"), int(nu)))


def tm_transfer_displacement(ctx: Ctx, u_full, points, out):
    """Old field u_full (3 Nn, this context's mesh) at the integer points (n, 3) int32 device
    tensor into out (3 n doubles, device)."""
    import torch
    n = int(points.shape[0])
    ctx.check(load_library().tm_transfer_displacement(ctx.handle, _vec(ctx, u_full, torch.float64, "u_full"), n,
                                                      _ptr(points, torch.int32, 3 * n, "points"),
                                                      _ptr(out, torch.float64, 3 * n, "out")))


# ---------------------------------------------------------------- learned initial guess
def _voxels(ctx: Ctx, g: int) -> int:
    i = ctx.mesh_desc
    return (i[0] << g) * (i[1] << g) * (i[2] << g)


def tm_learn_input(ctx: Ctx, rho, f, g, x) -> float:
    """Network input (4 channels on the level-g voxel grid) into x; returns the load scale s."""
    import torch
    s = C.c_double()
    ctx.check(load_library().tm_learn_input(ctx.handle, _elem(ctx, rho, "rho"), _vec(ctx, f, torch.float64, "f"),
                                            int(g), _ptr(x, torch.float32, 4 * _voxels(ctx, g), "x"), C.byref(s)))
    return s.value


def tm_learn_guess(ctx: Ctx, out, s, g, u0):
    import torch
    ctx.check(load_library().tm_learn_guess(ctx.handle, _ptr(out, torch.float32, 3 * _voxels(ctx, g), "out"),
                                            float(s), int(g), _vec(ctx, u0, torch.float64, "u0")))


def tm_learn_output_grad(ctx: Ctx, au0, f, s, g, dout):
    import torch
    ctx.check(load_library().tm_learn_output_grad(ctx.handle, _vec(ctx, au0, torch.float64, "au0"),
                                                  _vec(ctx, f, torch.float64, "f"), float(s), int(g),
                                                  _ptr(dout, torch.float32, 3 * _voxels(ctx, g), "dout")))


def tm_adam_step(ctx: Ctx, params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    import torch
    n = params.numel()
    ctx.check(load_library().tm_adam_step(ctx.handle, n, _ptr(params, torch.float32, n, "params"),
                                          _ptr(grads, torch.float32, n, "grads"), _ptr(m, torch.float32, n, "m"),
                                          _ptr(v, torch.float32, n, "v"), int(step), lr, beta1, beta2, eps))
