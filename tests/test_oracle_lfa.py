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


# ---- Definition 2.1 against the textbook smoothing factor of damped Jacobi
# On the 5-point (7-point) Laplacian the Jacobi symbol is 1 - w (1 - c), c the
# mean of cos(theta_a).  Over T_high at least one theta_a has cos <= 0, so c
# runs over [-1, 1/2] in 2D ([-1, 2/3] in 3D) and, S being affine in c,
#   mu = max(|1 - w/2|, |1 - 2w|)  (2D),   max(|1 - w/3|, |1 - 2w|)  (3D):
# the classic 3/5 at w = 4/5 (2D) and 5/7 at w = 6/7 (3D).  The sampled meshes
# contain the extremal frequencies (0, pi/2, pi) exactly.  A wrong high-frequency
# set (e.g. low frequencies included: c up to 1, mu -> 1) or a wrong supremum
# fails these.

@pytest.mark.parametrize("w,mu", [(0.8, 0.6), (0.5, 0.75), (1.0, 1.0), (0.6, 0.7), (2.0 / 3.0, 2.0 / 3.0)])
def test_mu_loc_jacobi_5_point_textbook(w, mu):
    lap = {(0, 0): 4.0, (1, 0): -1.0, (-1, 0): -1.0, (0, 1): -1.0, (0, -1): -1.0}
    assert abs(max(abs(1 - w / 2), abs(1 - 2 * w)) - mu) < 1e-15       # the closed form itself
    assert abs(lfa.mu_loc(lap, "jacobi", w, samples=256) - mu) < 1e-12


@pytest.mark.parametrize("w,mu", [(6.0 / 7.0, 5.0 / 7.0), (0.5, 5.0 / 6.0), (1.0, 1.0)])
def test_mu_loc_jacobi_7_point_textbook(w, mu):
    lap = {(0, 0, 0): 6.0}
    for a in range(3):
        for s in (-1, 1):
            off = [0, 0, 0]
            off[a] = s
            lap[tuple(off)] = -1.0
    assert abs(max(abs(1 - w / 3), abs(1 - 2 * w)) - mu) < 1e-15
    assert abs(lfa.mu_loc(lap, "jacobi", w, samples=48) - mu) < 1e-12


def test_mu_loc_is_over_high_frequencies_only():
    """The Jacobi symbol reaches 1 at theta = 0 (a low frequency): a supremum
    over all frequencies would give 1 for every w; Definition 2.1 excludes them."""
    lap = {(0, 0): 4.0, (1, 0): -1.0, (-1, 0): -1.0, (0, 1): -1.0, (0, -1): -1.0}
    th0 = np.zeros((1, 2))
    assert abs(lfa.smoother_symbol(lap, "jacobi", 0.8, th0)[0] - 1.0) < 1e-15
    assert lfa.mu_loc(lap, "jacobi", 0.8, samples=64) < 0.61


# ---- compact 4th-order stencils: symbols in closed form
def test_compact9_symbol_is_eq_hsymbol():
    """Eq. Hsymbol: a + 2b cos t1 + 2b cos t2 + 4c cos t1 cos t2 with the
    constants a, b, c of Section 4.1 (sigma as in Eq. 1)."""
    h, sigma = 1.0 / 64, 900.0 * (1 - 0.01j)
    st = operator.compact9_stencil(h, sigma)
    a = 10 / (3 * h ** 2) - 2 * sigma / 3
    b = -2 / (3 * h ** 2) - sigma / 12
    c = -1 / (6 * h ** 2)
    th = np.random.default_rng(3).uniform(-np.pi, np.pi, (200, 2))
    c1, c2 = np.cos(th[:, 0]), np.cos(th[:, 1])
    ref = a + 2 * b * c1 + 2 * b * c2 + 4 * c * c1 * c2
    assert np.allclose(lfa.symbol(st, th), ref, rtol=1e-13, atol=0)


def test_compact19_symbol_closed_form():
    """The 3D analogue of Eq. Hsymbol, summed by hand from the printed L and M
    of Eq. disc4thCompact3D: the 6 faces give 2 cos t_a per axis, the 12 edges
    4 cos t_a cos t_b per pair of axes, so
      H~ = -(1/6h^2)(-24 + 4 sum c_a + 4 sum_{a<b} c_a c_b) - sigma (6 + 2 sum c_a)/12."""
    h, sigma = 1.0 / 32, 400.0 * (1 - 0.01j)
    st = operator.compact19_stencil(h, sigma)
    assert len(st) == 19
    th = np.random.default_rng(4).uniform(-np.pi, np.pi, (200, 3))
    c = np.cos(th)
    s1 = c.sum(axis=1)
    s2 = c[:, 0] * c[:, 1] + c[:, 0] * c[:, 2] + c[:, 1] * c[:, 2]
    ref = -(-24 + 4 * s1 + 4 * s2) / (6 * h ** 2) - sigma * (6 + 2 * s1) / 12
    assert np.allclose(lfa.symbol(st, th), ref, rtol=1e-13, atol=0)
