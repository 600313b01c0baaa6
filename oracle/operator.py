"""Discrete acoustic Helmholtz operator (oracle; test infrastructure only).

Eq. (1):  -Lap p - omega^2 kappa^2 (1 - i gamma/omega) p = q.

Second-order finite differences (5-point 2D / 7-point 3D, Section 2.1) on a
nodal grid with h = 1/(n-1).  Boundary nodes carry the first-order absorbing
condition dp/dn = -i omega kappa p (outgoing waves for the sign of the
attenuation term in Eq. (1)) through a ghost point; each boundary row is then
multiplied by 1/2 per boundary axis, which makes the matrix complex symmetric
(A = A^T).  Written out, with per-axis weights w(i) = 1/2 at the two end nodes
and 1 elsewhere, and b(i) = 1 at the end nodes and 0 elsewhere:

  (A u)_p = sum_a [prod_{a'!=a} w_a'(p)] sum_{q = p +- e_a in grid} (u_p - u_q)/h^2
          + [prod_a w_a(p)] c_p u_p
          + (i omega kappa_p / h) sum_a b_a(p) [prod_{a'!=a} w_a'(p)] u_p,
  c_p = -omega^2 kappa_p^2 (1 - i gamma_p/omega).

The right-hand side is scaled the same way: q_hat = (prod_a w_a) q.

The shifted operator of Eq. (shift) adds i alpha omega^2 M with the lumped
(5-point) mass matrix M = diag(prod_a w_a); the sign is that of the
attenuation term, i.e. the shift adds damping (reading of Eq. shift).

Sparse matrices use the flattened index x + n_x*(y + n_y*z); with scipy's
kron(A, B) (row index i_A*n_B + i_B) the x factor is therefore the LAST
factor of each Kronecker product.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def axis_weights(n: int, periodic: bool = False):
    """Per-axis half-cell weights w and boundary indicators b (see module doc)."""
    w = np.ones(n)
    b = np.zeros(n)
    if not periodic:
        w[0] = w[-1] = 0.5
        b[0] = b[-1] = 1.0
    return w, b


def second_difference_1d(n: int, h: float, periodic: bool = False) -> sp.csr_matrix:
    """Row p: sum over the in-grid neighbours q of (u_p - u_q)/h^2."""
    if periodic:
        D = 2.0 * sp.eye(n, format="lil")
        for i in range(n):
            D[i, (i - 1) % n] += -1.0
            D[i, (i + 1) % n] += -1.0
        return (D.tocsr() / h ** 2).astype(np.float64)
    main = np.full(n, 2.0)
    main[0] = main[-1] = 1.0
    off = -np.ones(n - 1)
    return (sp.diags([off, main, off], [-1, 0, 1], format="csr") / h ** 2).astype(np.float64)


def _kron_axes(factors):
    """Kronecker product of per-axis factors given in axis order (x, y, z):
    the x factor is innermost (last)."""
    out = None
    for f in reversed(factors):
        out = f if out is None else sp.kron(out, f, format="csr")
    return sp.csr_matrix(out)


def mass_diagonal(shape_xyz, periodic: bool = False) -> np.ndarray:
    """prod_a w_a(p) per node (the lumped mass / row scaling), flattened."""
    ws = [sp.diags(axis_weights(n, periodic)[0]) for n in shape_xyz]
    return _kron_axes(ws).diagonal().copy()


def helmholtz(shape_xyz, h: float, kappa: np.ndarray, omega: float, gamma: np.ndarray,
              periodic: bool = False) -> sp.csr_matrix:
    """Assemble A of Eq. (1) (module doc).  shape_xyz = (n_x, n_y[, n_z]);
    kappa, gamma are per-node arrays (any shape with the right size, C order
    with x fastest)."""
    d = len(shape_xyz)
    kap = np.asarray(kappa, dtype=np.float64).ravel()
    gam = np.asarray(gamma, dtype=np.float64).ravel()
    W = [sp.diags(axis_weights(n, periodic)[0]) for n in shape_xyz]
    B = [sp.diags(axis_weights(n, periodic)[1]) for n in shape_xyz]
    Dm = [second_difference_1d(n, h, periodic) for n in shape_xyz]
    lap = None
    abc = None
    for a in range(d):
        lap_f = [Dm[k] if k == a else W[k] for k in range(d)]
        abc_f = [B[k] if k == a else W[k] for k in range(d)]
        t = _kron_axes(lap_f)
        s = _kron_axes(abc_f)
        lap = t if lap is None else lap + t
        abc = s if abc is None else abc + s
    wmass = mass_diagonal(shape_xyz, periodic)
    c = -omega ** 2 * kap ** 2 * (1.0 - 1j * gam / omega)
    diag = wmass * c + (1j * omega * kap / h) * abc.diagonal()
    A = lap.astype(np.complex128) + sp.diags(diag)
    return sp.csr_matrix(A)


def shifted(A: sp.csr_matrix, shape_xyz, omega: float, alpha: float,
            periodic: bool = False) -> sp.csr_matrix:
    """A_s = A + i alpha omega^2 M, M = lumped mass diag(prod_a w_a) (Eq. shift,
    sign read as added damping)."""
    M = mass_diagonal(shape_xyz, periodic)
    return sp.csr_matrix(A + sp.diags(1j * alpha * omega ** 2 * M))


def scaled_rhs(q: np.ndarray, shape_xyz, periodic: bool = False) -> np.ndarray:
    """q_hat = (prod_a w_a) q: the right-hand side of the row-scaled system."""
    return mass_diagonal(shape_xyz, periodic) * np.asarray(q).ravel()


# --------------------------------------------------------------------------
# Constant-coefficient stencils (used by the pins only)
# --------------------------------------------------------------------------

def stencil_matrix(shape_xyz, stencil: dict, periodic: bool = False) -> sp.csr_matrix:
    """Matrix of a constant stencil {offset (dx, dy[, dz]): value}; offsets that
    leave the grid are dropped (truncation) unless periodic."""
    d = len(shape_xyz)
    N = int(np.prod(shape_xyz))
    grids = np.meshgrid(*[np.arange(n) for n in reversed(shape_xyz)], indexing="ij")
    coords = [g.ravel() for g in reversed(grids)]          # x, y, z coordinate arrays
    idx = np.arange(N)
    rows, cols, vals = [], [], []
    for off, val in stencil.items():
        ok = np.ones(N, dtype=bool)
        nb = []
        for a in range(d):
            c = coords[a] + off[a]
            if periodic:
                c = c % shape_xyz[a]
            else:
                ok &= (c >= 0) & (c < shape_xyz[a])
            nb.append(c)
        flat = np.zeros(N, dtype=np.int64)
        stride = 1
        for a in range(d):
            flat += np.where(ok, nb[a], 0) * stride
            stride *= shape_xyz[a]
        rows.append(idx[ok])
        cols.append(flat[ok])
        vals.append(np.full(ok.sum(), val, dtype=np.complex128))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def five_point_stencil(h: float, sigma: complex, dim: int = 2) -> dict:
    """Interior 2nd-order stencil of Eq. (1): -Lap_h - sigma, sigma = kappa^2 omega^2 (1 - i gamma/omega)."""
    st = {tuple([0] * dim): 2.0 * dim / h ** 2 - sigma}
    for a in range(dim):
        for s in (-1, 1):
            off = [0] * dim
            off[a] = s
            st[tuple(off)] = -1.0 / h ** 2
    return st


def compact9_stencil(h: float, sigma: complex) -> dict:
    """Compact 4th-order 2D stencil, Eq. (disc4thCompact): L/h^2 - sigma*M."""
    L = {(0, 0): 10 / 3, (1, 0): -2 / 3, (-1, 0): -2 / 3, (0, 1): -2 / 3, (0, -1): -2 / 3,
         (1, 1): -1 / 6, (1, -1): -1 / 6, (-1, 1): -1 / 6, (-1, -1): -1 / 6}
    M = {(0, 0): 2 / 3, (1, 0): 1 / 12, (-1, 0): 1 / 12, (0, 1): 1 / 12, (0, -1): 1 / 12}
    st = {k: v / h ** 2 for k, v in L.items()}
    for k, v in M.items():
        st[k] = st[k] - sigma * v
    return st


def compact19_stencil(h: float, sigma: complex) -> dict:
    """Compact 3D stencil, Eq. (disc4thCompact3D): L - sigma*M with
    L = -1/(6h^2) * {centre -24, 6 face neighbours 2, 12 edge neighbours 1}
    (the 8 corners are zero: 19 points) and M = 1/12 * {centre 6, faces 1}."""
    st = {}
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                m = abs(dx) + abs(dy) + abs(dz)
                if m == 0:
                    lv = -24.0
                elif m == 1:
                    lv = 2.0
                elif m == 2:
                    lv = 1.0
                else:
                    continue
                st[(dx, dy, dz)] = -lv / (6.0 * h ** 2)
    st[(0, 0, 0)] -= sigma * 6.0 / 12.0
    for a in range(3):
        for s in (-1, 1):
            off = [0, 0, 0]
            off[a] = s
            st[tuple(off)] -= sigma * 1.0 / 12.0
    return st


# --------------------------------------------------------------------------
# Compact fourth-order operator (Eqs. disc4thCompact, disc4thCompact3D)
# --------------------------------------------------------------------------
# The printed stencils are H = L - sigma M for a constant sigma =
# kappa^2 omega^2 (1 - i gamma/omega) (Eq. 1's coefficient; Section 2.1).
# Readings for a variable medium and the boundary (the paper is silent):
#   - sigma varies per node: H = L - (Sigma M + M Sigma)/2, Sigma = diag(sigma):
#     complex symmetric, the printed stencil wherever sigma is constant, fourth
#     order there and second order where sigma varies;
#   - boundary: the stencils are applied at every node with the neighbours
#     outside the grid dropped (homogeneous Dirichlet truncation); absorption
#     comes from the attenuation layer of the medium (gamma), not from a
#     boundary condition;
#   - right-hand side q_hat = M q (the mass stencil applied to the source, as
#     the fourth-order compact scheme requires);
#   - shift (Eq. shift with M the compact mass stencil): A_s = A + i alpha omega^2 M.

def compact_parts(shape_xyz, h: float, periodic: bool = False):
    """(L, M): the matrices of the compact Laplacian stencil (divided by h^2)
    and of the compact mass stencil, truncated at the boundary."""
    d = len(shape_xyz)
    st0 = compact9_stencil(h, 0.0) if d == 2 else compact19_stencil(h, 0.0)
    # the printed mass stencils, written out (not recovered as a difference of
    # two stencils, which would lose digits against the 1/h^2 entries)
    mass = {tuple([0] * d): 2.0 / 3.0 if d == 2 else 6.0 / 12.0}
    for a in range(d):
        for sgn in (-1, 1):
            off = [0] * d
            off[a] = sgn
            mass[tuple(off)] = 1.0 / 12.0
    return (stencil_matrix(shape_xyz, st0, periodic).real.astype(np.float64),
            stencil_matrix(shape_xyz, mass, periodic).real.astype(np.float64))


def helmholtz_compact(shape_xyz, h: float, kappa: np.ndarray, omega: float, gamma: np.ndarray,
                      periodic: bool = False) -> sp.csr_matrix:
    """H = L - (Sigma M + M Sigma)/2 (readings above)."""
    L, M = compact_parts(shape_xyz, h, periodic)
    kap = np.asarray(kappa, dtype=np.float64).ravel()
    gam = np.asarray(gamma, dtype=np.float64).ravel()
    S = sp.diags(omega ** 2 * kap ** 2 * (1.0 - 1j * gam / omega))
    return sp.csr_matrix(L.astype(np.complex128) - 0.5 * (S @ M + M @ S))


def shifted_compact(A: sp.csr_matrix, shape_xyz, h: float, omega: float, alpha: float,
                    periodic: bool = False) -> sp.csr_matrix:
    """A_s = A + i alpha omega^2 M with the compact mass stencil M."""
    _, M = compact_parts(shape_xyz, h, periodic)
    return sp.csr_matrix(A + 1j * alpha * omega ** 2 * M)


def scaled_rhs_compact(q: np.ndarray, shape_xyz, h: float, periodic: bool = False) -> np.ndarray:
    """q_hat = M q."""
    _, M = compact_parts(shape_xyz, h, periodic)
    return M @ np.asarray(q, dtype=np.complex128).ravel()
