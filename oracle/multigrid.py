"""Shifted-Laplacian multigrid hierarchy and V-cycle (oracle; test infrastructure only).

Section 2.3 / 3.1: the preconditioner is multigrid applied to the shifted
operator H_s (Eq. shift); coarse operators are Galerkin products
A_{l+1} = R_l A_l P_l (Section 3.1) with the intergrid scheme of
`transfer.scheme_kinds`.  Algorithm 1 (two-grid cycle) with step 3 replaced by
a recursive call gives the V-cycle, by two recursive calls the W-cycle
(Section 2.2); the coarsest level is
solved exactly by LU with partial pivoting (SuperLU; an exact direct solve).
Coarse initial guesses are zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import defaults, transfer, vanka


@dataclass
class Level:
    shape: tuple            # (n_x, n_y[, n_z])
    A: sp.csr_matrix        # shifted operator on this level
    M: sp.csr_matrix | None = None     # assembled Vanka sum (None on the coarsest)
    w: float = 1.0          # damping
    R: sp.csr_matrix | None = None     # restriction to the next level
    P: sp.csr_matrix | None = None     # prolongation from the next level
    lu: object | None = None           # LU factors of A (coarsest level only)


def build_hierarchy(A_s: sp.csr_matrix, shape_xyz, levels: int, patches, scheme: str,
                    damping=None, periodic: bool = False):
    """Galerkin hierarchy of `levels` levels for the shifted operator A_s.

    patches: one patch kind per smoothed level (levels-1 entries) or a single
    kind for all; damping: matching list, default the paper's table."""
    d = len(shape_xyz)
    if isinstance(patches, str):
        patches = [patches] * (levels - 1)
    if damping is None:
        damping = [defaults.damping(d, patches[l], l) for l in range(levels - 1)]
    out = []
    A = sp.csr_matrix(A_s)
    shape = tuple(shape_xyz)
    for l in range(levels):
        if l == levels - 1:
            order = "MMD_ATA" if periodic else "MMD_AT_PLUS_A"      # fill-reducing ordering only
            lu = spla.splu(sp.csc_matrix(A), permc_spec=order, diag_pivot_thresh=1.0)
            out.append(Level(shape=shape, A=A, lu=lu))
            break
        M = vanka.smoother_matrix(A, shape, patches[l], periodic)
        rk, pk = transfer.scheme_kinds(scheme, l)
        shape_c = transfer.coarse_shape(shape, periodic)
        R = transfer.restriction(shape_c, rk, periodic)
        P = transfer.prolongation(shape_c, pk, periodic)
        out.append(Level(shape=shape, A=A, M=M, w=damping[l], R=R, P=P))
        A = sp.csr_matrix(R @ A @ P)
        shape = shape_c
    return out


def vcycle(hier, f: np.ndarray, level: int = 0, nu1: int = 1, nu2: int = 1,
           u: np.ndarray | None = None, cycle: str = "V") -> np.ndarray:
    """One V(nu1, nu2) or W(nu1, nu2) cycle for A_level u = f (Algorithm 1,
    applied recursively).  V: step 3 is one cycle on the coarser level; W: step
    3 is two cycles on the coarser level, the second starting from the first
    one's result (Section 2.2).  On the coarsest level a cycle is the exact
    solve, whatever the initial guess."""
    L = hier[level]
    if L.lu is not None:
        return L.lu.solve(np.asarray(f, dtype=np.complex128))
    u = np.zeros_like(f) if u is None else u.copy()
    for _ in range(nu1):                                   # step 1: pre-relaxation
        u = vanka.sweep(L.A, L.M, L.w, u, f)
    r_c = L.R @ (f - L.A @ u)                              # step 2: restrict residual
    e_c = vcycle(hier, r_c, level + 1, nu1, nu2, cycle=cycle)   # step 3: coarse problem (recursive)
    if cycle == "W":
        e_c = vcycle(hier, r_c, level + 1, nu1, nu2, u=e_c, cycle=cycle)
    elif cycle != "V":
        raise ValueError(cycle)
    u = u + L.P @ e_c                                      # step 4: coarse-grid correction
    for _ in range(nu2):                                   # step 5: post-relaxation
        u = vanka.sweep(L.A, L.M, L.w, u, f)
    return u


def operator_complexity(matrices) -> float:
    """Eq. (operatorComplexity): sum_l nnz(H^l) / nnz(H^1)."""
    nnz = [m.nnz for m in matrices]
    return sum(nnz) / nnz[0]


def convergence_factor(hier, u0: np.ndarray, f: np.ndarray, warmup: int = 5, target: float = 1e-9,
                       max_iter: int = 300, nu1: int = 1, nu2: int = 1) -> float:
    """Eq. (cf): c_f = (||r_k|| / ||r_0||)^(1/k) for the cycle used as a
    stationary solver u <- u + V(f - A u), counting from after `warmup`
    iterations until the relative residual (to the initial one) drops below
    `target` (Section 5.1)."""
    A = hier[0].A
    u = u0.astype(np.complex128).copy()
    r = f - A @ u
    rinit = np.linalg.norm(r)
    for _ in range(warmup):
        u = u + vcycle(hier, r, 0, nu1, nu2)
        r = f - A @ u
    r0 = np.linalg.norm(r)
    k = 0
    rk = r0
    while k < max_iter and rk / rinit > target:
        u = u + vcycle(hier, r, 0, nu1, nu2)
        r = f - A @ u
        rk = np.linalg.norm(r)
        k += 1
    return (rk / r0) ** (1.0 / k) if k > 0 else 0.0
