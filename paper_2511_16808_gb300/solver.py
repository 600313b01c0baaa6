"""Convenience layer over the C ABI: fills hz_grid / hz_opts from problem
parameters and runs setup / solve on torch CUDA tensors.  All computation
happens in libhz.so."""
from __future__ import annotations

import numpy as np
import torch

from . import hz


class HelmholtzSolver:
    """One hierarchy (hz_setup) for a medium, frequency and shift.

    kappa, gamma: per-node float64 arrays (numpy or torch, any device),
    flattened x-fastest.  patch: fine-level patch; patch_coarse: patch on the
    coarser levels (default: the same).  damping: per-level list, default the
    paper's table for each level's patch.  cycle: "V" or "W" (two cycles on
    the next level per visit, Section 2.2)."""

    def __init__(self, dim, n, kappa, omega, gamma, alpha, levels, patch="rb", intergrid="leveldep",
                 precision="mixed", tol=1e-6, restart=5, nu1=1, nu2=1, max_iter=2000,
                 patch_coarse=None, damping=None, nrhs_max=1, stream=None, cycle="V"):
        n = list(n) if hasattr(n, "__len__") else [n] * dim
        self.dim = dim
        self.n = n + [1] * (3 - len(n))
        self.nodes = int(np.prod(n[:dim]))
        self.h = 1.0 / (n[0] - 1)
        self.grid = hz.make_grid(dim, n, self.h)
        o = make_opts(dim, levels, patch=patch, intergrid=intergrid, precision=precision, tol=tol,
                      restart=restart, nu1=nu1, nu2=nu2, max_iter=max_iter, patch_coarse=patch_coarse,
                      damping=damping, nrhs_max=nrhs_max, cycle=cycle)
        self.opts = o
        self.mixed = precision == "mixed"
        self.stream = stream
        k = _as_f64(kappa)
        g = _as_f64(gamma) if gamma is not None else None
        self.ctx = hz.hz_setup(self.grid, k, omega, g, 0.0, alpha, o, stream)

    def solve(self, q, p=None):
        """q: complex128 source (unscaled), device or host; returns (p, info)."""
        if p is None:
            dev = q.device if isinstance(q, torch.Tensor) else "cuda"
            p = torch.empty(self.nodes, dtype=torch.complex128, device=dev)
        ok, infos = hz.hz_solve(self.ctx, q, p, 1, self.stream)
        return p, infos[0]

    def solve_batch(self, Q, P=None):
        """Q: complex128 [nodes, R] sources (RHS innermost), R a power of two
        <= nrhs_max; returns (P, [info] * R)."""
        R = Q.shape[1]
        if P is None:
            P = torch.empty_like(Q)
        ok, infos = hz.hz_solve(self.ctx, Q, P, R, self.stream)
        return P, infos

    def precond(self, r):
        z = torch.empty_like(r)
        nrhs = r.shape[1] if r.dim() == 2 else 1
        hz.hz_precond_apply(self.ctx, r, z, nrhs, self.stream)
        return z

    def apply(self, v, shifted=False):
        w = torch.empty_like(v)
        nrhs = v.shape[1] if v.dim() == 2 else 1
        hz.hz_apply_operator(self.ctx, v, w, nrhs, int(shifted), self.stream)
        return w

    def close(self):
        if getattr(self, "ctx", None):
            hz.hz_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def make_opts(dim, levels, patch="rb", intergrid="leveldep", precision="mixed", tol=1e-6, restart=5, nu1=1,
              nu2=1, max_iter=2000, patch_coarse=None, damping=None, nrhs_max=1, cycle="V") -> hz.hz_opts:
    """hz_opts from solver settings; damping defaults to the paper's table per
    level and patch."""
    o = hz.hz_opts_default(dim)
    o.levels = levels
    for l in range(hz.MAX_LEVELS):
        p = patch if l == 0 else (patch_coarse or patch)
        o.patch[l] = hz.PATCH[p]
        o.damping[l] = damping[l] if damping is not None and l < len(damping) \
            else hz.hz_default_damping(dim, p, l)
    o.nu1, o.nu2 = nu1, nu2
    o.intergrid = hz.INTERGRID[intergrid]
    o.precision = hz.PRECISION[precision]
    o.restart_m = restart
    o.tol = tol
    o.max_iter = max_iter
    o.nrhs_max = nrhs_max
    o.cycle_visits = {"V": 1, "W": 2}[cycle]
    return o


def _as_f64(a):
    if isinstance(a, torch.Tensor):
        return a.detach().to(torch.float64).contiguous().reshape(-1)
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
