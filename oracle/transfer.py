"""Intergrid operators (oracle; test infrastructure only).

Section 3.1.  The 1D factors are
  linear  (Eq. biliniearIntergrid):  R = [1 2 1]/4,      P = 2 R^T
  cubic   (Eq. bicubicIntergrid):    R = [1 4 6 4 1]/16, P = 2 R^T
and the d-dimensional operators are their Kronecker products
(Eqs. trilin, tricub), so that P = 2^d R^T (Section 3.1, after
Eq. bicubicIntergrid).  Coarse node k is fine node 2k; a grid of n_c coarse
nodes per axis has n_f = 2(n_c - 1) + 1 fine nodes (2 n_c when periodic).

Prolongation, 1D, coarse values c_k:
  linear: fine 2k <- c_k,                         fine 2k+1 <- (c_k + c_{k+1})/2
  cubic:  fine 2k <- 3/4 c_k + 1/8 (c_{k-1}+c_{k+1}), fine 2k+1 <- (c_k + c_{k+1})/2
At the two ends the cubic rule needs c_{-1} and c_{n_c}, which the paper does
not define; they are mirrored (c_{-1} := c_1, c_{n_c} := c_{n_c - 2}), which
keeps constants exact.  The restriction is always R_1D = P_1D^T / 2.

Intergrid schemes between level l and l+1 (l = 1 is the finest):
  'linear'   R_lin,  P_lin  on every level
  'cubic'    R_cub,  P_cub  on every level
  'mixed'    R_lin,  P_cub  on every level          (Section 5.2)
  'leveldep' R_cub,  P_cub  for 1->2 (Eq. level1Intergrid),
             R_lin,  P_cub  for k->k+1, k > 1 (Eq. levelDepIntergrid)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def prolong_1d(nc: int, kind: str, periodic: bool = False) -> sp.csr_matrix:
    """1D prolongation (n_f x n_c) of the given kind ('linear' or 'cubic')."""
    nf = 2 * nc if periodic else 2 * (nc - 1) + 1
    P = sp.lil_matrix((nf, nc))

    def add(i, k, v):
        if periodic:
            P[i % nf, k % nc] += v
        else:
            if 0 <= i < nf:
                if k < 0:          # mirrored ghost c_{-1} := c_1
                    k = 1
                elif k > nc - 1:   # mirrored ghost c_{nc} := c_{nc-2}
                    k = nc - 2
                P[i, k] += v

    for k in range(nc):
        if kind == "linear":
            add(2 * k, k, 1.0)
            if periodic or k + 1 < nc:
                add(2 * k + 1, k, 0.5)
                add(2 * k + 1, k + 1, 0.5)
        elif kind == "cubic":
            add(2 * k, k, 0.75)
            add(2 * k, k - 1, 0.125)
            add(2 * k, k + 1, 0.125)
            if periodic or k + 1 < nc:
                add(2 * k + 1, k, 0.5)
                add(2 * k + 1, k + 1, 0.5)
        else:
            raise ValueError(kind)
    return P.tocsr()


def restrict_1d(nc: int, kind: str, periodic: bool = False) -> sp.csr_matrix:
    """R_1D = P_1D^T / 2."""
    return sp.csr_matrix(prolong_1d(nc, kind, periodic).T / 2.0)


def _kron_axes(factors):
    out = None
    for f in reversed(factors):
        out = f if out is None else sp.kron(out, f, format="csr")
    return sp.csr_matrix(out)


def coarse_shape(shape_xyz, periodic: bool = False):
    if periodic:
        return tuple(n // 2 for n in shape_xyz)
    return tuple((n - 1) // 2 + 1 for n in shape_xyz)


def prolongation(shape_c_xyz, kind: str, periodic: bool = False) -> sp.csr_matrix:
    return _kron_axes([prolong_1d(n, kind, periodic) for n in shape_c_xyz])


def restriction(shape_c_xyz, kind: str, periodic: bool = False) -> sp.csr_matrix:
    return _kron_axes([restrict_1d(n, kind, periodic) for n in shape_c_xyz])


def scheme_kinds(scheme: str, level: int):
    """(restriction kind, prolongation kind) between level and level+1
    (level 0 is the finest grid)."""
    if scheme == "linear":
        return "linear", "linear"
    if scheme == "cubic":
        return "cubic", "cubic"
    if scheme == "mixed":
        return "linear", "cubic"
    if scheme == "leveldep":
        return ("cubic", "cubic") if level == 0 else ("linear", "cubic")
    raise ValueError(scheme)
