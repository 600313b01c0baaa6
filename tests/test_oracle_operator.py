"""Pins for the oracle's discrete operator (Eq. 1, Section 2.1; Eq. shift).

- A = A^T exactly (the symmetric half-cell boundary form).
- Interior rows equal the textbook 5-/7-point stencil built independently.
- Manufactured solutions converge at the second-order rate: an interior
  Gaussian-modulated wave with variable kappa (pins the Laplacian scaling
  and the sign of the mass and attenuation terms), and a plane wave meeting
  the absorbing condition with Robin data on every face (pins the ABC rows,
  their 1/h factor and the half-cell weighting, corners included).
- The shift sign: with the literal sign of Eq. (shift) the preconditioned
  solve stalls, with the damping sign it converges (reading of Eq. shift).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import operator, solver


def _kappa_gamma(shape, seed=0):
    rng = np.random.default_rng(seed)
    k = 0.5 + rng.random(int(np.prod(shape)))
    g = 0.5 * rng.random(int(np.prod(shape)))
    return k, g


@pytest.mark.parametrize("shape", [(9, 9), (7, 5), (5, 5, 5), (4, 6, 5)])
def test_operator_complex_symmetric(shape):
    k, g = _kappa_gamma(shape)
    A = operator.helmholtz(shape, 0.1, k, 7.0, g)
    assert abs(A - A.T).max() == 0.0
    As = operator.shifted(A, shape, 7.0, 0.3)
    assert abs(As - As.T).max() == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_interior_rows_are_textbook_stencil(dim):
    n = 7
    shape = (n,) * dim
    h, omega, kap, gam = 0.125, 9.0, 0.8, 0.4
    A = operator.helmholtz(shape, h, np.full(n ** dim, kap), omega, np.full(n ** dim, gam))
    sigma = kap ** 2 * omega ** 2 * (1 - 1j * gam / omega)
    S = operator.stencil_matrix(shape, operator.five_point_stencil(h, sigma, dim))
    co = np.stack(np.meshgrid(*[np.arange(n)] * dim, indexing="ij"), -1).reshape(-1, dim)
    interior = np.all((co > 0) & (co < n - 1), axis=1)
    D = (A - S).tocsr()[interior]
    assert abs(D).max() < 1e-9 * abs(S).max()
    # row sums of the Laplacian part vanish everywhere except via the mass/ABC diagonal
    assert np.count_nonzero(A[interior].getnnz(axis=1) != 2 * dim + 1) == 0


def _grid(n, dim):
    t = np.linspace(0.0, 1.0, n)
    g = np.meshgrid(*([t] * dim), indexing="ij")      # [z][y][x] ordering
    return [x.ravel() for x in reversed(g)]           # x, y[, z] coordinate vectors


def _mms_bump_error(n, dim, omega, gamma):
    """Max nodal error for u = exp(-|x-c|^2/(2 s^2)) exp(i k.x), variable kappa."""
    h = 1.0 / (n - 1)
    X = _grid(n, dim)
    s, kv = 0.07 if dim == 2 else 0.09, np.array([13.0, -7.0, 5.0][:dim])
    dx = [x - 0.5 for x in X]
    r2 = sum(d * d for d in dx)
    u = np.exp(-r2 / (2 * s * s)) * np.exp(1j * sum(kv[a] * X[a] for a in range(dim)))
    lap = (-dim / s ** 2 + r2 / s ** 4 - 2j * sum(kv[a] * dx[a] for a in range(dim)) / s ** 2
           - kv @ kv) * u
    kappa = 1.0 + 0.2 * np.sin(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[1])
    f = -lap - omega ** 2 * kappa ** 2 * (1 - 1j * gamma / omega) * u
    shape = (n,) * dim
    A = operator.helmholtz(shape, h, kappa, omega, np.full(n ** dim, gamma))
    lu = spla.splu(sp.csc_matrix(A), permc_spec="MMD_AT_PLUS_A")
    uh = lu.solve(operator.scaled_rhs(f, shape))
    return np.max(np.abs(uh - u))


def test_mms_interior_second_order_2d():
    errs = [_mms_bump_error(n, 2, 20.0, 2.0) for n in (33, 65, 129, 257)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8) and np.all(rates < 2.3), rates


def test_mms_interior_second_order_3d():
    errs = [_mms_bump_error(n, 3, 6.0, 1.0) for n in (9, 17, 33)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 1.8 and rates[-1] < 2.4, rates


def _mms_plane_wave_error(n, phi, omega, gamma):
    """Plane wave u = exp(-i omega (x cos phi + y sin phi)), kappa = 1, with the
    ghost-point Robin data g = du/dn + i omega u on every face added to the
    right-hand side (weight of the face's other axis, times 1/h)."""
    h = 1.0 / (n - 1)
    x, y = _grid(n, 2)
    d = np.array([np.cos(phi), np.sin(phi)])
    u = np.exp(-1j * omega * (d[0] * x + d[1] * y))
    f = -(-omega ** 2) * u - omega ** 2 * (1 - 1j * gamma / omega) * u   # -Lap u - sigma u
    shape = (n, n)
    A = operator.helmholtz(shape, h, np.ones(n * n), omega, np.full(n * n, gamma))
    rhs = operator.scaled_rhs(f, shape)
    i = np.rint(x / h).astype(int)
    j = np.rint(y / h).astype(int)
    wx = np.where((i == 0) | (i == n - 1), 0.5, 1.0)
    wy = np.where((j == 0) | (j == n - 1), 0.5, 1.0)
    for mask, normal, wother in (((i == 0), (-1, 0), wy), ((i == n - 1), (1, 0), wy),
                                 ((j == 0), (0, -1), wx), ((j == n - 1), (0, 1), wx)):
        g = 1j * omega * (1.0 - d @ np.array(normal)) * u     # du/dn + i omega u
        rhs = rhs + np.where(mask, wother * g / h, 0.0)
    uh = spla.spsolve(sp.csc_matrix(A), rhs)
    return np.max(np.abs(uh - u))


@pytest.mark.parametrize("phi", [0.0, np.pi / 6, np.pi / 4])
def test_mms_absorbing_boundary_second_order(phi):
    errs = [_mms_plane_wave_error(n, phi, 15.0, 1.5) for n in (33, 65, 129, 257)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), rates


def test_shift_sign_reading():
    """Eq. (shift) prints -i alpha omega^2 M; the attenuation of Eq. (1) is
    +i gamma omega kappa^2.  A shift that removes damping stalls the solve;
    the damping sign converges (the reading used throughout)."""
    n = 65
    h = 1.0 / (n - 1)
    omega = 2 * np.pi / (10 * h)
    shape = (n, n)
    q = np.zeros(n * n, complex)
    q[(n // 2) * n + n // 2] = 1 / h ** 2
    kw = dict(shape_xyz=shape, h=h, kappa=np.ones(n * n), omega=omega,
              gamma=np.full(n * n, 0.01 * omega), levels=3, patch="plus", scheme="leveldep")
    _, good = solver.Problem(alpha=0.25, **kw).solve(q, tol=1e-7, max_iter=200)
    _, bad = solver.Problem(alpha=-0.25, **kw).solve(q, tol=1e-7, max_iter=200)
    assert good.converged and good.iters < 80
    assert not bad.converged or bad.iters > 2 * good.iters


# ---- compact 4th-order stencils (Eqs. disc4thCompact, disc4thCompact3D) ----
# Both are "Mehrstellen" discretisations: applied to a smooth u they give
#   (L - sigma M) u = (I + h^2/12 Lap_h)(-Lap u - sigma u) + O(h^4),
# with Lap_h the textbook 5-/7-point Laplacian, i.e. M = I + h^2/12 Lap_h and
# L u = -Lap u - (h^2/12) Lap^2 u + O(h^4).  The stencils are even, so the
# O(h^4) remainder holds only 6th derivatives: on polynomials of degree <= 5
# the identity is exact (up to rounding).  The right side is built from the
# analytic Laplacian and the textbook 2nd-order stencil only, so a wrong
# centre, face, edge or mass weight of the printed stencils fails it.

def _rand_poly(dim, deg, rng):
    """{exponent tuple: coefficient} of a random polynomial of total degree <= deg."""
    import itertools
    return {e: rng.standard_normal() for e in itertools.product(range(deg + 1), repeat=dim) if sum(e) <= deg}


def _poly_eval(p, x):
    return sum(c * np.prod([xi ** ei for xi, ei in zip(x, e)]) for e, c in p.items())


def _poly_lap(p):
    """Analytic Laplacian of the polynomial."""
    out = {}
    for e, c in p.items():
        for a in range(len(e)):
            if e[a] >= 2:
                f = list(e)
                f[a] -= 2
                out[tuple(f)] = out.get(tuple(f), 0.0) + c * e[a] * (e[a] - 1)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_compact_stencils_fourth_order_identity(dim):
    rng = np.random.default_rng(11 + dim)
    for trial in range(4):
        h = [0.1, 0.05, 0.2, 0.125][trial]
        sigma = complex(rng.uniform(5, 50), rng.uniform(-1, 0))
        st = operator.compact9_stencil(h, sigma) if dim == 2 else operator.compact19_stencil(h, sigma)
        p = _rand_poly(dim, 5, rng)
        x0 = rng.uniform(-1, 1, dim)
        lhs = sum(v * _poly_eval(p, x0 + h * np.asarray(off, float)) for off, v in st.items())
        lap = _poly_lap(p)
        g = lambda x: -_poly_eval(lap, x) - sigma * _poly_eval(p, x)       # -Lap u - sigma u
        lap_h = sum(g(x0 + h * np.eye(dim)[a] * s) for a in range(dim) for s in (-1, 1)) - 2 * dim * g(x0)
        rhs = g(x0) + lap_h / 12.0                                            # h^2/12 Lap_h g, Lap_h = (...)/h^2
        scale = max(abs(lhs), abs(g(x0)), 1.0)
        assert abs(lhs - rhs) <= 1e-9 * scale * (1 + abs(sigma)), (dim, trial, lhs, rhs)


@pytest.mark.parametrize("dim", [2, 3])
def test_compact_stencils_not_fourth_order_on_degree_six(dim):
    """The same identity fails on x^6 (a 6th-derivative term remains), so the
    test above is not vacuous."""
    h, sigma = 0.1, 0.0
    st = operator.compact9_stencil(h, sigma) if dim == 2 else operator.compact19_stencil(h, sigma)
    p = {tuple([6] + [0] * (dim - 1)): 1.0}
    x0 = np.zeros(dim)
    lhs = sum(v * _poly_eval(p, x0 + h * np.asarray(off, float)) for off, v in st.items())
    lap = _poly_lap(p)
    g = lambda x: -_poly_eval(lap, x)
    lap_h = sum(g(x0 + h * np.eye(dim)[a] * s) for a in range(dim) for s in (-1, 1)) - 2 * dim * g(x0)
    assert abs(lhs - (g(x0) + lap_h / 12.0)) > 1e-3 * h ** 4


@pytest.mark.parametrize("dim", [2, 3])
def test_compact_stencils_row_sums(dim):
    """L annihilates constants and M sums to one (the mass of a node)."""
    st0 = operator.compact9_stencil(0.1, 0.0) if dim == 2 else operator.compact19_stencil(0.1, 0.0)
    st1 = operator.compact9_stencil(0.1, 1.0) if dim == 2 else operator.compact19_stencil(0.1, 1.0)
    assert abs(sum(st0.values())) < 1e-10
    assert abs(sum(st0.values()) - sum(st1.values()) - 1.0) < 1e-12
