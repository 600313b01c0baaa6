"""Flexible GMRES(m) with right preconditioning (oracle; test infrastructure only).

Section 2.3 uses the shifted-Laplacian cycle as a preconditioner inside
(flexible) GMRES; Section 5.2 fixes the restart length m = 5.  One restart
cycle, from the current iterate x with residual r = b - A x, beta = ||r||:
  v_0 = r / beta;  g = beta e_0
  for j = 0..m-1:
      z_j = M(v_j)                      (preconditioner application; counted)
      w = A z_j
      for i = 0..j:  h_ij = v_i^H w;  w -= h_ij v_i     (modified Gram-Schmidt)
      h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j}
      apply the previous complex Givens rotations to column j of H, form the
      rotation that zeroes h_{j+1,j}, apply it to g
      stop the cycle if |g_{j+1}| / ||b|| < tol
  y = H[:k,:k]^{-1} g[:k];  x += Z[:k] y;  r = b - A x (true residual)
and the solve ends when ||r|| / ||b|| < tol.  The iteration count is the
number of preconditioner applications.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Info:
    iters: int = 0
    relres_est: float = np.inf
    relres_true: float = np.inf
    converged: bool = False
    history: list = field(default_factory=list)   # |g_{j+1}| / ||b|| per iteration


def givens(a: complex, b: complex):
    """Complex rotation G = [[c, s], [-conj(s), c]] (c real) with G [a, b]^T = [rho, 0]^T."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def fgmres(A, b: np.ndarray, precond, m: int = 5, tol: float = 1e-6, max_iter: int = 1000,
           x0: np.ndarray | None = None):
    """Solve A x = b.  A: callable or matrix; precond: callable v -> z."""
    matvec = A if callable(A) else (lambda v: A @ v)
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = np.linalg.norm(b)
    info = Info()
    if bnorm == 0:
        info.converged, info.relres_est, info.relres_true = True, 0.0, 0.0
        return np.zeros(n, dtype=np.complex128), info
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    info.relres_true = beta / bnorm
    if info.relres_true < tol:
        info.converged = True
        return x, info
    while info.iters < max_iter:
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            info.iters += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            info.relres_est = abs(g[j + 1]) / bnorm
            info.history.append(info.relres_est)
            if info.relres_est < tol or info.iters >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Z[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        info.relres_true = beta / bnorm
        if info.relres_true < tol:
            info.converged = True
            break
    return x, info
