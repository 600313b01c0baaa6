"""Pins for the oracle's FGMRES(m) (Section 2.3) and V-cycle (Algorithm 1, Eq. 2G).

FGMRES
- With a fixed linear preconditioner Mp, after j <= m iterations of the first
  cycle the iterate minimises ||b - A x|| over x in Mp K_j(A Mp, b); checked
  against a dense least-squares solve over an explicitly built Krylov basis
  (no Arnoldi), both for the residual estimate and the true residual.
- An exact preconditioner converges in one iteration.
- Restarted FGMRES reaches the tolerance and the dense solution.
- A complex Givens rotation is unitary and zeroes the second entry.
V-cycle
- The two-level cycle's error propagation equals
  S^nu2 (I - P A_c^{-1} R A) S^nu1 with S = I - w M A, built from dense
  matrices (Eq. 2G); the coarse-grid correction is a projection.
- The cycle is linear in its right-hand side.
- V- and W-cycles over 3 and 4 levels: the error propagation equals the
  textbook recursion E_l = S^nu2 (I - P (I - E_{l+1}^g) A_{l+1}^{-1} R A) S^nu1
  with E_coarsest = 0 and g = 1 (V) or 2 (W) cycles on the coarser level
  (Section 2.2; Trottenberg, Oosterlee & Schueller, Multigrid, Sec. 2.4),
  built from dense matrices; a two-level W-cycle equals the V-cycle.
"""
import numpy as np
import pytest

from oracle import fgmres, multigrid, operator, solver


def _random_system(n=40, seed=0, shift=3.0, mp_scale=0.2):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * shift + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Mp = np.eye(n) + mp_scale * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, Mp, b


@pytest.mark.parametrize("j", [1, 2, 3, 4, 5])
def test_fgmres_minimises_residual_over_krylov_space(j):
    A, Mp, b = _random_system()
    x, info = fgmres.fgmres(A, b, lambda v: Mp @ v, m=5, tol=1e-30, max_iter=j)
    assert info.iters == j
    K = np.zeros((b.size, j), complex)
    v = b.copy()
    for k in range(j):
        K[:, k] = v
        v = A @ (Mp @ v)
    X = Mp @ K
    c, *_ = np.linalg.lstsq(A @ X, b, rcond=None)
    best = np.linalg.norm(b - A @ X @ c) / np.linalg.norm(b)
    assert np.isclose(info.relres_true, best, rtol=1e-8)
    assert np.isclose(info.relres_est, best, rtol=1e-8)


def test_exact_preconditioner_converges_in_one_iteration():
    A, _, b = _random_system()
    Ainv = np.linalg.inv(A)
    x, info = fgmres.fgmres(A, b, lambda v: Ainv @ v, m=5, tol=1e-10)
    assert info.iters == 1 and info.converged
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10)


def test_restarted_fgmres_reaches_dense_solution():
    A, Mp, b = _random_system(60, seed=2, shift=25.0, mp_scale=0.02)
    x, info = fgmres.fgmres(A, b, lambda v: Mp @ v, m=5, tol=1e-11, max_iter=2000)
    assert info.converged and info.iters > 5
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-11
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-8)


def test_givens_rotation():
    rng = np.random.default_rng(4)
    for _ in range(20):
        a, b = rng.standard_normal(2) @ np.array([1, 1j]), rng.standard_normal(2) @ np.array([1, 1j])
        c, s = fgmres.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        assert np.allclose(G.conj().T @ G, np.eye(2), atol=1e-14)
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-14 * abs(out[0])


def _small_problem(levels=2, patch="plus", scheme="leveldep", n=9):
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(5)
    N = n * n
    return solver.Problem((n, n), h, 0.7 + 0.6 * rng.random(N), 11.0, 0.2 * rng.random(N) + 0.1,
                          0.3, levels, patch, scheme)


@pytest.mark.parametrize("patch", ["plus", "element", "rb", "jacobi"])
@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (0, 1)])
def test_two_level_error_propagation_is_eq_2g(patch, nu):
    pr = _small_problem(2, patch)
    pr.nu1, pr.nu2 = nu
    L0, L1 = pr.hier
    A = L0.A.toarray()
    N = A.shape[0]
    S = np.eye(N) - L0.w * L0.M.toarray() @ A
    P, R = L0.P.toarray(), L0.R.toarray()
    Ac = R @ A @ P
    assert np.allclose(Ac, L1.A.toarray(), rtol=1e-12, atol=1e-9)
    CGC = np.eye(N) - P @ np.linalg.solve(Ac, R @ A)
    TG = np.linalg.matrix_power(S, nu[1]) @ CGC @ np.linalg.matrix_power(S, nu[0])
    B = np.column_stack([pr.precond(np.eye(N)[:, j].astype(complex)) for j in range(N)])
    assert np.allclose(np.eye(N) - B @ A, TG, atol=1e-9)
    assert np.allclose(CGC @ CGC, CGC, atol=1e-9)


def test_vcycle_is_linear():
    pr = _small_problem(3, "plus", n=17)
    rng = np.random.default_rng(7)
    N = 17 * 17
    f, g = (rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N)))
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    assert np.allclose(pr.precond(a * f + b * g), a * pr.precond(f) + b * pr.precond(g), atol=1e-10)


def _dense_cycle_error(hier, level, nu, g):
    L = hier[level]
    A = L.A.toarray()
    N = A.shape[0]
    if L.lu is not None:
        return np.zeros((N, N), dtype=complex)
    S = np.eye(N) - L.w * L.M.toarray() @ A
    P, R = L.P.toarray(), L.R.toarray()
    Ac = hier[level + 1].A.toarray()
    Ec = _dense_cycle_error(hier, level + 1, nu, g)
    inner = np.eye(Ac.shape[0]) - np.linalg.matrix_power(Ec, g)
    CGC = np.eye(N) - P @ inner @ np.linalg.solve(Ac, R @ A)
    return np.linalg.matrix_power(S, nu[1]) @ CGC @ np.linalg.matrix_power(S, nu[0])


@pytest.mark.parametrize("levels", [3, 4])
@pytest.mark.parametrize("cycle,g", [("V", 1), ("W", 2)])
@pytest.mark.parametrize("nu", [(1, 1), (2, 1)])
def test_multilevel_error_propagation_recursion(levels, cycle, g, nu):
    pr = _small_problem(levels, "rb", n=17)
    pr.nu1, pr.nu2 = nu
    pr.cycle = cycle
    A = pr.hier[0].A.toarray()
    N = A.shape[0]
    B = np.column_stack([pr.precond(np.eye(N)[:, j].astype(complex)) for j in range(N)])
    E = _dense_cycle_error(pr.hier, 0, nu, g)
    assert np.allclose(np.eye(N) - B @ A, E, atol=1e-9)


def test_two_level_w_cycle_is_v_cycle():
    pr = _small_problem(2, "plus")
    rng = np.random.default_rng(3)
    f = rng.standard_normal(81) + 1j * rng.standard_normal(81)
    zv = pr.precond(f)
    pr.cycle = "W"
    assert np.array_equal(pr.precond(f), zv)
    pr3 = _small_problem(3, "plus", n=17)
    f3 = rng.standard_normal(289) + 1j * rng.standard_normal(289)
    zv3 = pr3.precond(f3)
    pr3.cycle = "W"
    assert np.linalg.norm(pr3.precond(f3) - zv3) > 1e-6 * np.linalg.norm(zv3)   # a real difference
