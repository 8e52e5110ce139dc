"""Shared set-up of the GPU parity tests: one library context, workloads uploaded
to it, and the oracle's view of the same problem."""
import functools

import numpy as np

import workloads as W
from oracle import fem as F
from oracle import mesh as M

U32 = np.finfo(np.float32).eps
U64 = np.finfo(np.float64).eps


@functools.lru_cache(maxsize=None)
def tm():
    from paper_1009_4975_gb300 import build
    build.build()
    import paper_1009_4975_gb300 as P
    P.load_library()
    return P


@functools.lru_cache(maxsize=None)
def ctx():
    import torch
    torch.cuda.init()
    return tm().tm_create(0, stream=torch.cuda.current_stream())


class Case:
    """A workload uploaded to the library together with the oracle's reduced system."""

    def __init__(self, w, assemble=True):
        import torch
        self.w = w
        d = w.dom
        self.m = M.build_mesh(d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, dirichlet_faces=w.dirichlet_faces)
        self.rho = w.rho[self.m.perm].copy()
        if assemble:
            self.A, self.f, self.C = F.reduced_system(self.m, self.rho, w.load_nodes, w.load_comp, w.load_val,
                                                      w.E0, w.Emin, w.nu, w.penal)
        self.fn = F.free_nodes(self.m)
        self.dev = torch.device("cuda:0")

    def direct(self):
        """The oracle's direct solution of the reduced system, computed once per case."""
        if getattr(self, "_ud", None) is None:
            from oracle import solve as S
            self._ud = S.direct(self.A, self.f)
        return self._ud

    def upload(self):
        w, d = self.w, self.w.dom
        info = tm().tm_mesh_upload(ctx(), d.nx, d.ny, d.nz, d.L, d.h0, w.leaves, w.dirichlet_faces, w.E0, w.Emin,
                                   w.nu, w.penal)
        return info

    def t(self, a, dtype=None):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device=self.dev)

    def full(self, v_free):
        return F.to_full_layout(self.m, v_free)

    def free(self, v_full):
        return F.from_full_layout(self.m, v_full)


@functools.lru_cache(maxsize=None)
def case(name):
    makers = {"config1": W.config1, "config1b": W.config1b, "small_truss": W.small_truss,
              "truss_10x5x5_L1": lambda: W.truss_mesh("truss_10x5x5_L1", W.Domain(10, 5, 5, 1, 0.2), 3, r0=0.06)}
    return Case(makers[name]())
