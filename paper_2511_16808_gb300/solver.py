"""Convenience layer over the C ABI: fills hz_grid / hz_opts from problem
parameters and runs setup / solve on torch CUDA tensors.  All computation
happens in libhz.so."""
from __future__ import annotations

import json
import time

import numpy as np
import torch

from . import hz


class JsonLines:
    """Append-only JSON-lines sink: a path (opened in append mode) or an open
    text file; one object per line, flushed after each."""

    def __init__(self, target):
        self._own = isinstance(target, str)
        self._f = open(target, "a", encoding="utf-8") if self._own else target

    def write(self, record: dict):
        self._f.write(json.dumps(record, sort_keys=True) + "\n")
        self._f.flush()

    def close(self):
        if self._own and self._f:
            self._f.close()
        self._f = None


def solve_record(kind, infos, history, setup_s, wall_s, nodes, opts_desc):
    """The per-solve metrics line: iterations, convergence, true residual,
    the restart history (single-RHS solves), setup and solve wall time."""
    its = [i.iters for i in infos]
    rec = {"event": kind, "t": time.time(), "nodes": nodes, "nrhs": len(infos), "iters": its,
           "converged": [bool(i.converged) for i in infos], "relres_true": [i.relres_true for i in infos],
           "relres_est": [i.relres_est for i in infos], "setup_s": setup_s, "wall_s": wall_s,
           "vcycles": int(sum(its)), "solves_per_s": (len(infos) / wall_s) if wall_s > 0 else None}
    if history is not None:
        rec["history"] = history
    rec.update(opts_desc)
    return rec


class HelmholtzSolver:
    """One hierarchy (hz_setup) for a medium, frequency and shift.

    kappa, gamma: per-node float64 arrays (numpy or torch, any device),
    flattened x-fastest.  patch: fine-level patch; patch_coarse: patch on the
    coarser levels (default: the same).  damping: per-level list, default the
    paper's table for each level's patch.  cycle: "V" or "W" (two cycles on
    the next level per visit, Section 2.2).  stencil: "second" (5-/7-point)
    or "compact" (the fourth-order stencils of Section 2.1).  log: a path or text file that
    receives one JSON line per solve (solve_record)."""

    def __init__(self, dim, n, kappa, omega, gamma, alpha, levels, patch="rb", intergrid="leveldep",
                 precision="mixed", tol=1e-6, restart=5, nu1=1, nu2=1, max_iter=2000,
                 patch_coarse=None, damping=None, nrhs_max=1, stream=None, cycle="V", log=None,
                 stencil="second"):
        n = list(n) if hasattr(n, "__len__") else [n] * dim
        self.dim = dim
        self.n = n + [1] * (3 - len(n))
        self.nodes = int(np.prod(n[:dim]))
        self.h = 1.0 / (n[0] - 1)
        self.grid = hz.make_grid(dim, n, self.h)
        o = make_opts(dim, levels, patch=patch, intergrid=intergrid, precision=precision, tol=tol,
                      restart=restart, nu1=nu1, nu2=nu2, max_iter=max_iter, patch_coarse=patch_coarse,
                      damping=damping, nrhs_max=nrhs_max, cycle=cycle, stencil=stencil)
        self.opts = o
        self.mixed = precision == "mixed"
        self.stream = stream
        k = _as_f64(kappa)
        g = _as_f64(gamma) if gamma is not None else None
        self.ctx = hz.hz_setup(self.grid, k, omega, g, 0.0, alpha, o, stream)
        self.log = JsonLines(log) if log is not None else None
        self._desc = {"dim": dim, "n": n[:dim], "levels": levels, "patch": patch,
                      "patch_coarse": patch_coarse or patch, "intergrid": intergrid, "precision": precision,
                      "tol": tol, "restart": restart, "cycle": cycle, "alpha": alpha, "omega": omega,
                      "stencil": stencil}

    def _log(self, kind, infos, t0, single):
        if self.log is None:
            return
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        hist = hz.hz_solve_history(self.ctx) if single else None
        self.log.write(solve_record(kind, infos, hist, hz.hz_setup_seconds(self.ctx), wall, self.nodes,
                                    self._desc))

    def solve(self, q, p=None):
        """q: complex128 source (unscaled), device or host; returns (p, info)."""
        if p is None:
            dev = q.device if isinstance(q, torch.Tensor) else "cuda"
            p = torch.empty(self.nodes, dtype=torch.complex128, device=dev)
        t0 = time.perf_counter()
        ok, infos = hz.hz_solve(self.ctx, q, p, 1, self.stream)
        self._log("solve", infos, t0, True)
        return p, infos[0]

    def solve_batch(self, Q, P=None):
        """Q: complex128 [nodes, R] sources (RHS innermost), R a power of two
        <= nrhs_max; returns (P, [info] * R)."""
        R = Q.shape[1]
        if P is None:
            P = torch.empty_like(Q)
        t0 = time.perf_counter()
        ok, infos = hz.hz_solve(self.ctx, Q, P, R, self.stream)
        self._log("solve_batch", infos, t0, R == 1)
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

    def setup_seconds(self) -> float:
        return hz.hz_setup_seconds(self.ctx)

    def history(self) -> dict:
        """Iterations, true and estimated relative residual at the start and
        after every restart cycle of the last single-RHS solve."""
        return hz.hz_solve_history(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            hz.hz_destroy(self.ctx)
            self.ctx = None
        if getattr(self, "log", None):
            self.log.close()
            self.log = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def make_opts(dim, levels, patch="rb", intergrid="leveldep", precision="mixed", tol=1e-6, restart=5, nu1=1,
              nu2=1, max_iter=2000, patch_coarse=None, damping=None, nrhs_max=1, cycle="V",
              stencil="second") -> hz.hz_opts:
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
    o.stencil = {"second": 0, "compact": 1}[stencil]
    return o


def _as_f64(a):
    if isinstance(a, torch.Tensor):
        return a.detach().to(torch.float64).contiguous().reshape(-1)
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
