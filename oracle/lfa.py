"""Local Fourier analysis (oracle side tool; test infrastructure only).

Section 4 of the paper.  Everything here is written from the symbol formulas
and is independent of the matrix code in `operator`, `transfer` and `vanka`,
so that it can pin that code (on periodic grids LFA is exact).

  H~(theta)  symbol of a constant stencil {offset d: s_d}: sum_d s_d e^{i theta.d}
             (for the compact 9-point stencil this is Eq. Hsymbol)
  S~(theta)  additive Vanka smoother symbol, Eq. (smoother_symbol):
             1 - w (V^T W Phi^H H_i^{-1} Phi V) H~(theta), with V = ones(N),
             W = I/N, Phi = diag(e^{i theta.d_k}) over the patch offsets d_k,
             (H_i)_{kl} = s_{d_l - d_k} (Eqs. 4lfa, 5lfa, skew5lfa)
  R~(theta)  restriction symbol, per axis (1 + cos t)/2 for the linear and
             (3 + 4 cos t + cos 2t)/8 for the cubic stencil (Section 4.2)
  TG~(theta) two-grid symbol on the 4 (2D) / 8 (3D) harmonics, Eq. (symbolTG):
             S~^nu2 (I - P~ H~_c^{-1} R~ H~) S~^nu1, H~_c = R~ H~ P~ (Galerkin)
  mu_loc     Definition 2.1: sup over T_high of |S~|
  rho_loc    Definition 2.2: sup over T_low of rho(TG~)
"""
from __future__ import annotations

import itertools

import numpy as np

# Patch offsets as printed in the diagonal of Phi (Eqs. 4lfa, 5lfa, skew5lfa);
# 3D patches follow the definitions of Section 3.2.
PATCHES_2D = {
    "element": [(0, 0), (1, 0), (0, 1), (1, 1)],
    "plus": [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)],
    "rb": [(-1, -1), (1, -1), (0, 0), (-1, 1), (1, 1)],
    "full": [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
    "jacobi": [(0, 0)],
}


def patch_offsets_lfa(kind: str, dim: int):
    if dim == 2:
        return PATCHES_2D[kind]
    box = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    if kind == "element":
        return [(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    if kind == "plus":
        return [o for o in box if sum(map(abs, o)) <= 1]
    if kind == "rb":
        return [o for o in box if sum(map(abs, o)) % 2 == 0]
    if kind == "full":
        return box
    if kind == "jacobi":
        return [(0, 0, 0)]
    raise ValueError(kind)


def symbol(stencil: dict, theta: np.ndarray) -> np.ndarray:
    """H~(theta) for theta of shape (..., d)."""
    out = np.zeros(theta.shape[:-1], dtype=np.complex128)
    for off, s in stencil.items():
        out = out + s * np.exp(1j * (theta @ np.asarray(off, dtype=np.float64)))
    return out


def patch_matrix(stencil: dict, offsets) -> np.ndarray:
    """(H_i)_{kl} = s_{d_l - d_k}: the constant-coefficient patch matrix."""
    N = len(offsets)
    H = np.zeros((N, N), dtype=np.complex128)
    for k, dk in enumerate(offsets):
        for l, dl in enumerate(offsets):
            H[k, l] = stencil.get(tuple(b - a for a, b in zip(dk, dl)), 0.0)
    return H


def smoother_symbol(stencil: dict, kind: str, w: float, theta: np.ndarray) -> np.ndarray:
    """S~(theta), Eq. (smoother_symbol), for theta of shape (..., d)."""
    dim = theta.shape[-1]
    offs = patch_offsets_lfa(kind, dim)
    N = len(offs)
    Hinv = np.linalg.inv(patch_matrix(stencil, offs))
    D = np.asarray(offs, dtype=np.float64)                 # (N, d)
    phi = np.exp(1j * (theta @ D.T))                      # (..., N): diagonal of Phi
    # V^T W Phi^H Hinv Phi V = (1/N) sum_{k,l} conj(phi_k) Hinv_kl phi_l
    m = np.einsum("...k,kl,...l->...", np.conj(phi), Hinv, phi) / N
    return 1.0 - w * m * symbol(stencil, theta)


def restriction_symbol(kind: str, theta: np.ndarray) -> np.ndarray:
    """R~(theta) (Section 4.2): product of the per-axis symbols."""
    out = np.ones(theta.shape[:-1])
    for a in range(theta.shape[-1]):
        t = theta[..., a]
        if kind == "linear":
            out = out * (1.0 + np.cos(t)) / 2.0
        elif kind == "cubic":
            out = out * (3.0 + 4.0 * np.cos(t) + np.cos(2.0 * t)) / 8.0
        else:
            raise ValueError(kind)
    return out


def harmonics(theta: np.ndarray) -> np.ndarray:
    """The 2^d harmonics theta + pi*alpha, alpha in {0,1}^d (Definition 2.3);
    returns (..., 2^d, d), the first being theta itself."""
    dim = theta.shape[-1]
    shifts = np.array(list(itertools.product((0, 1), repeat=dim)), dtype=np.float64) * np.pi
    return theta[..., None, :] + shifts


def two_grid_symbol(stencil: dict, kind: str, w: float, rk: str, pk: str, theta: np.ndarray,
                    nu1: int = 1, nu2: int = 1) -> np.ndarray:
    """TG~(theta) of Eq. (symbolTG); theta (..., d) -> (..., 2^d, 2^d)."""
    th = harmonics(theta)
    Hd = symbol(stencil, th)                               # (..., K)
    Sd = smoother_symbol(stencil, kind, w, th)             # (..., K)
    Rr = restriction_symbol(rk, th)                        # (..., K) row of R~
    Pc = restriction_symbol(pk, th)                        # (..., K) column of P~
    Hc = np.sum(Rr * Hd * Pc, axis=-1)                     # (...) Galerkin coarse symbol
    K = Hd.shape[-1]
    eye = np.eye(K)
    cgc = eye - (Pc[..., :, None] / Hc[..., None, None]) * (Rr * Hd)[..., None, :]
    S = Sd[..., :, None] * eye
    TG = cgc
    for _ in range(nu1):
        TG = TG @ S
    for _ in range(nu2):
        TG = S @ TG
    return TG


def low_frequencies(samples: int, dim: int) -> np.ndarray:
    """Uniform samples of T_low = [-pi/2, pi/2)^d, shape (samples^d, d)."""
    t = -np.pi / 2 + np.pi * np.arange(samples) / samples
    g = np.meshgrid(*([t] * dim), indexing="ij")
    return np.stack([x.ravel() for x in g], axis=-1)


def rho_loc(stencil, kind, w, rk, pk, samples: int = 128, nu1: int = 1, nu2: int = 1,
            theta: np.ndarray | None = None) -> float:
    """Definition 2.2: sup over (sampled) T_low of the spectral radius of TG~."""
    dim = len(next(iter(stencil)))
    th = low_frequencies(samples, dim) if theta is None else theta
    TG = two_grid_symbol(stencil, kind, w, rk, pk, th, nu1, nu2)
    return float(np.max(np.abs(np.linalg.eigvals(TG))))


def mu_loc(stencil, kind, w, samples: int = 256) -> float:
    """Definition 2.1: sup over T_high of |S~| (sampled on a samples^d mesh of
    [-pi/2, 3pi/2)^d)."""
    dim = len(next(iter(stencil)))
    t = -np.pi / 2 + 2 * np.pi * np.arange(samples) / samples
    g = np.meshgrid(*([t] * dim), indexing="ij")
    th = np.stack([x.ravel() for x in g], axis=-1)
    high = np.any(th >= np.pi / 2, axis=-1)
    return float(np.max(np.abs(smoother_symbol(stencil, kind, w, th[high]))))
