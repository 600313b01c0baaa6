"""Oracle solver facade (test infrastructure only).

Puts the pieces together as the paper's method: the Helmholtz operator A of
Eq. (1), the shifted operator A_s of Eq. (shift), the Galerkin multigrid
hierarchy of A_s with additive Vanka smoothing (Sections 3.1-3.3), one
V(nu1, nu2) (or W) cycle (Algorithm 1, recursive) as the preconditioner, and
FGMRES(m) on the row-scaled system A p = q_hat (Section 2.3, m = 5 in
Section 5.2), zero initial guess (Section 5).  stencil="compact" takes the
compact fourth-order stencils of Section 2.1 instead of the 5-/7-point one.
"""
from __future__ import annotations

import numpy as np

from . import fgmres as _fgmres
from . import multigrid, operator


class Problem:
    def __init__(self, shape_xyz, h, kappa, omega, gamma, alpha, levels, patch, scheme,
                 patch_coarse=None, nu1=1, nu2=1, damping=None, periodic=False, cycle="V",
                 stencil="second"):
        self.shape = tuple(shape_xyz)
        self.h = h
        self.omega = omega
        self.nu1, self.nu2 = nu1, nu2
        self.cycle = cycle
        self.periodic = periodic
        self.stencil = stencil
        if stencil == "compact":      # Eqs. disc4thCompact(3D), readings in operator.py
            self.A = operator.helmholtz_compact(self.shape, h, kappa, omega, gamma, periodic)
            self.A_s = operator.shifted_compact(self.A, self.shape, h, omega, alpha, periodic)
        else:
            self.A = operator.helmholtz(self.shape, h, kappa, omega, gamma, periodic)
            self.A_s = operator.shifted(self.A, self.shape, omega, alpha, periodic)
        patches = [patch] + [patch_coarse or patch] * (levels - 2)
        self.hier = multigrid.build_hierarchy(self.A_s, self.shape, levels, patches[: levels - 1],
                                              scheme, damping, periodic)

    def precond(self, r: np.ndarray) -> np.ndarray:
        """z = V- (or W-) cycle(r) with zero initial guess."""
        return multigrid.vcycle(self.hier, np.asarray(r, dtype=np.complex128), 0, self.nu1, self.nu2,
                                cycle=self.cycle)

    def rhs(self, q: np.ndarray) -> np.ndarray:
        if self.stencil == "compact":
            return operator.scaled_rhs_compact(q, self.shape, self.h, self.periodic)
        return operator.scaled_rhs(q, self.shape, self.periodic)

    def solve(self, q: np.ndarray, tol: float, m: int = 5, max_iter: int = 2000):
        """FGMRES(m) for A p = q_hat from p = 0; returns (p, info)."""
        return _fgmres.fgmres(self.A, self.rhs(q), self.precond, m=m, tol=tol, max_iter=max_iter)


def from_workload(w, **overrides) -> Problem:
    """Problem for a `workloads.Workload`."""
    kw = dict(shape_xyz=w.shape, h=w.h, kappa=w.kappa, omega=w.omega, gamma=w.gamma,
              alpha=w.alpha, levels=w.levels, patch=w.patch, scheme=w.intergrid,
              patch_coarse=w.patch_coarse, nu1=w.nu1, nu2=w.nu2, cycle=w.cycle)
    kw.update(overrides)
    return Problem(**kw)
