"""Additive Vanka smoother (oracle; test infrastructure only).

Section 3.2: with X_i the node set of patch i and V_i the injection onto it,
the patch matrix is H_i = V_i H V_i^T and one additive sweep is
  u <- u + w * sum_i V_i^T W_i H_i^{-1} V_i (q - H u)          (Eq. smoother)
where all patches see the same residual.  Patches (Section 3.2, offsets
about the patch anchor, written (dx, dy[, dz])):
  element  the 2^d vertices of a cell (anchor = lower corner of each cell)
  plus     the anchor and its 2d nearest neighbours
  rb       the anchor and the nodes of its red-black colour in the 3^d box
           (an X of 5 nodes in 2D, 13 nodes in 3D)
  full     the 3^d box
  jacobi   the anchor alone (a 1x1 patch: damped Jacobi, Section 4.1)
Boundary treatment (Section 3.3): for every patch type except the element
patch, patches are anchored at every node and clipped to the domain (the
intersection of the patch with the grid); every node j gets the weight
1/(number of patches containing j), and (W_i)_jj is that weight.  Element
patches are anchored at cells only and are never partial.

The sum in Eq. (smoother) is assembled once per level into one sparse
matrix M = sum_i V_i^T W_i H_i^{-1} V_i, so that a sweep is u += w M r.
H_i^{-1} is computed by LAPACK (LU with partial pivoting) through
numpy.linalg.inv.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def patch_offsets(kind: str, dim: int):
    """Offsets of one patch, as a list of d-tuples."""
    box = list(itertools.product((-1, 0, 1), repeat=dim))
    if kind == "element":
        return [tuple(reversed(t)) for t in itertools.product((0, 1), repeat=dim)]
    if kind == "plus":
        out = [tuple([0] * dim)]
        for a in range(dim):
            for s in (-1, 1):
                o = [0] * dim
                o[a] = s
                out.append(tuple(o))
        return out
    if kind == "rb":
        return [tuple(reversed(t)) for t in box if sum(abs(v) for v in t) % 2 == 0]
    if kind == "full":
        return [tuple(reversed(t)) for t in box]
    if kind == "jacobi":
        return [tuple([0] * dim)]
    raise ValueError(kind)


def _coords(shape_xyz):
    """x, y[, z] coordinate arrays of all nodes in flattened order."""
    grids = np.meshgrid(*[np.arange(n) for n in reversed(shape_xyz)], indexing="ij")
    return [g.ravel() for g in reversed(grids)]


def patch_index_table(shape_xyz, kind: str, periodic: bool = False) -> np.ndarray:
    """(n_patches, N) array of the node indices of each patch; -1 where the
    patch leaves the grid (clipped boundary patches).  Patches left with no
    node are not listed."""
    d = len(shape_xyz)
    offs = patch_offsets(kind, d)
    co = _coords(shape_xyz)
    if kind == "element" and not periodic:
        ok = np.ones(co[0].size, dtype=bool)
        for a in range(d):
            ok &= co[a] < shape_xyz[a] - 1
        anchors = [c[ok] for c in co]
    else:
        anchors = co
    P = anchors[0].size
    table = np.full((P, len(offs)), -1, dtype=np.int64)
    for k, off in enumerate(offs):
        inside = np.ones(P, dtype=bool)
        flat = np.zeros(P, dtype=np.int64)
        stride = 1
        for a in range(d):
            c = anchors[a] + off[a]
            if periodic:
                c = c % shape_xyz[a]
            else:
                inside &= (c >= 0) & (c < shape_xyz[a])
            flat += np.where(inside, c, 0) * stride
            stride *= shape_xyz[a]
        table[:, k] = np.where(inside, flat, -1)
    return table[(table >= 0).any(axis=1)]


def node_weights(table: np.ndarray, N: int) -> np.ndarray:
    """Section 3.3: weight of node j = 1 / (number of patches containing j)."""
    count = np.bincount(table[table >= 0], minlength=N).astype(np.float64)
    if (count == 0).any():
        raise ValueError("patches do not cover every node")
    return 1.0 / count


def _entries(A: sp.csr_matrix, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """A[rows[t], cols[t]] for every t (zero where not stored)."""
    return np.asarray(A[rows, cols]).ravel()


def patch_matrices(A: sp.csr_matrix, table: np.ndarray):
    """Group the patches by their valid-node pattern and return, per group,
    (patch row numbers, valid slot numbers, H_i stacked (g, m, m)) with
    H_i = V_i A V_i^T."""
    valid = table >= 0
    keys, inverse = np.unique(valid, axis=0, return_inverse=True)
    groups = []
    for gi, key in enumerate(keys):
        rows = np.nonzero(inverse.ravel() == gi)[0]
        slots = np.nonzero(key)[0]
        idx = table[np.ix_(rows, slots)]                  # (g, m) node indices
        m = slots.size
        r = np.repeat(idx, m, axis=1).ravel()             # row node of entry (k, l)
        c = np.tile(idx, (1, m)).ravel()                  # column node of entry (k, l)
        H = _entries(A, r, c).reshape(rows.size, m, m)
        groups.append((rows, slots, H))
    return groups


def smoother_matrix(A: sp.csr_matrix, shape_xyz, kind: str, periodic: bool = False) -> sp.csr_matrix:
    """M = sum_i V_i^T W_i H_i^{-1} V_i (Eq. smoother without the damping w)."""
    N = A.shape[0]
    table = patch_index_table(shape_xyz, kind, periodic)
    wt = node_weights(table, N)
    R, C, V = [], [], []
    for rows, slots, H in patch_matrices(A, table):
        Hinv = np.linalg.inv(H)                           # LU with partial pivoting
        idx = table[np.ix_(rows, slots)]
        m = slots.size
        r = np.repeat(idx, m, axis=1).ravel()
        c = np.tile(idx, (1, m)).ravel()
        R.append(r)
        C.append(c)
        V.append(wt[r] * Hinv.ravel())
    M = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(N, N))
    return sp.csr_matrix(M)


def sweep(A: sp.csr_matrix, M: sp.csr_matrix, w: float, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """One additive Vanka relaxation, Eq. (smoother): u + w M (f - A u)."""
    return u + w * (M @ (f - A @ u))
