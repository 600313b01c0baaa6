"""Pins tying the oracle's cycle to the paper's local Fourier analysis (Section 4).

- The Jacobi smoother symbol (a 1x1 Vanka patch, Section 4.1) equals the
  textbook damped-Jacobi symbol 1 - w H~/s_0.
- On small periodic grids LFA is exact: the eigenvalues of the oracle's
  two-grid error operator (dense, column by column) equal the union of the
  eigenvalues of the two-grid symbols TG~(theta) (Eq. symbolTG) over the
  grid's low frequencies.  This pins the smoother, the transfers, the
  Galerkin coarse operator and the cycle structure at once.
- Section 5.1 procedure: the measured convergence factor c_f (Eq. cf) of the
  two-grid cycle as a solver on a periodic homogeneous 256^2-cell grid, zero
  right-hand side, random initial guess, matches rho_loc (Definition 2.2)
  within 0.02 for each patch, with the damping of Table relaxParam.
"""
import numpy as np
import pytest

from oracle import defaults, lfa, multigrid, operator, solver


def _periodic_setup(n, ppw=10.0, gamma_over_omega=0.01):
    h = 1.0 / n
    omega = 2 * np.pi / (ppw * h)
    gamma = gamma_over_omega * omega
    sigma = omega ** 2 * (1 - 1j * gamma / omega)
    return h, omega, gamma, sigma


def test_jacobi_symbol_is_textbook():
    h, omega, gamma, sigma = _periodic_setup(64)
    st = operator.five_point_stencil(h, sigma, 2)
    th = np.random.default_rng(1).uniform(-np.pi / 2, 3 * np.pi / 2, (100, 2))
    w = 0.8
    ref = 1 - w * lfa.symbol(st, th) / st[(0, 0)]
    assert np.allclose(lfa.smoother_symbol(st, "jacobi", w, th), ref, atol=1e-13)


def _dense_two_grid(pr):
    A = pr.A_s.toarray()
    N = A.shape[0]
    B = np.zeros((N, N), complex)
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1.0
        B[:, j] = pr.precond(e)
    return np.eye(N) - B @ A


@pytest.mark.parametrize("patch", ["jacobi", "element", "plus", "rb", "full"])
@pytest.mark.parametrize("scheme,kinds", [("cubic", ("cubic", "cubic")), ("mixed", ("linear", "cubic")),
                                          ("linear", ("linear", "linear"))])
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_lfa_is_exact_on_periodic_grid(patch, scheme, kinds, alpha):
    n = 16
    h, omega, gamma, sigma = _periodic_setup(n, ppw=6.0)
    w = 0.7
    pr = solver.Problem((n, n), h, np.ones(n * n), omega, np.full(n * n, gamma), alpha, 2, patch,
                        scheme, damping=[w], periodic=True)
    ev_dense = np.sort(np.abs(np.linalg.eigvals(_dense_two_grid(pr))))
    st = operator.five_point_stencil(h, sigma - 1j * alpha * omega ** 2, 2)
    k = np.arange(-n // 4, n // 4)
    th = np.stack(np.meshgrid(2 * np.pi * k / n, 2 * np.pi * k / n, indexing="ij"), -1).reshape(-1, 2)
    TG = lfa.two_grid_symbol(st, patch, w, kinds[0], kinds[1], th)
    ev_lfa = np.sort(np.abs(np.linalg.eigvals(TG)).ravel())
    assert ev_dense.size == ev_lfa.size
    assert np.allclose(ev_dense, ev_lfa, atol=1e-9)


@pytest.mark.parametrize("patch", ["element", "plus", "rb", "jacobi"])
def test_measured_cf_matches_rho_loc(patch):
    n = 256
    h, omega, gamma, sigma = _periodic_setup(n)
    w = defaults.damping(2, patch, 0)
    st = operator.five_point_stencil(h, sigma, 2)
    rho = lfa.rho_loc(st, patch, w, "cubic", "cubic", samples=128)
    pr = solver.Problem((n, n), h, np.ones(n * n), omega, np.full(n * n, gamma), 0.0, 2, patch,
                        "cubic", periodic=True)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    cf = multigrid.convergence_factor(pr.hier, u0, np.zeros(n * n, complex))
    assert abs(cf - rho) <= 0.02, (patch, cf, rho)
