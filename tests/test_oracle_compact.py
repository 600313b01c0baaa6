"""Pins of the oracle's compact fourth-order operator (Section 2.1, Eqs.
disc4thCompact and disc4thCompact3D, with the readings stated in
oracle/operator.py for a variable medium, the boundary and the right-hand
side).

- Interior rows in a constant medium are the printed stencils L - sigma M
  (2D and 3D), sigma = kappa^2 omega^2 (1 - i gamma/omega) of Eq. 1.
- The operator is complex symmetric (A = A^T) in a variable medium too.
- Manufactured solution, constant medium, smooth compactly supported bump:
  the error of A u_h = M f falls at the fourth-order rate (2D and 3D); in a
  variable medium at least at the second-order rate of the symmetric
  (Sigma M + M Sigma)/2 form.
- The shift adds i alpha omega^2 M with the compact mass stencil, and the
  right-hand side is M q.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import operator


def _grid(n, dim):
    x = np.linspace(0.0, 1.0, n)
    g = np.meshgrid(*([x] * dim), indexing="ij")
    return [gi.transpose() for gi in g]            # arrays indexed [z][y][x] (x fastest when raveled)


@pytest.mark.parametrize("dim", [2, 3])
def test_interior_rows_are_printed_stencils(dim):
    n, h = 7, 1.0 / 6
    omega, gamma = 20.0, 0.3
    sigma = omega ** 2 * (1 - 1j * gamma / omega)
    shape = (n,) * dim
    A = operator.helmholtz_compact(shape, h, np.ones(n ** dim), omega, np.full(n ** dim, gamma))
    st = operator.compact9_stencil(h, sigma) if dim == 2 else operator.compact19_stencil(h, sigma)
    c = tuple([n // 2] * dim)
    p = int(np.ravel_multi_index(tuple(reversed(c)), tuple(reversed(shape))))
    row = A.getrow(p).toarray().ravel()
    for off, v in st.items():
        q = int(np.ravel_multi_index(tuple(reversed([c[a] + off[a] for a in range(dim)])), tuple(reversed(shape))))
        assert abs(row[q] - v) <= 1e-12 * abs(v), (off, row[q], v)
    assert np.count_nonzero(np.abs(row) > 0) == len([v for v in st.values() if v != 0])


@pytest.mark.parametrize("dim", [2, 3])
def test_compact_operator_complex_symmetric(dim):
    n = 9 if dim == 2 else 6
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(5)
    kappa = rng.uniform(0.3, 1.0, n ** dim)
    gamma = rng.uniform(0.0, 5.0, n ** dim)
    A = operator.helmholtz_compact((n,) * dim, h, kappa, 30.0, gamma)
    assert abs(A - A.T).max() == 0.0
    As = operator.shifted_compact(A, (n,) * dim, h, 30.0, 0.4)
    _, M = operator.compact_parts((n,) * dim, h)
    assert abs((As - A) - 1j * 0.4 * 900.0 * M).max() < 1e-9
    q = np.zeros(n ** dim, complex)
    q[n ** dim // 2] = 1.0
    assert np.allclose(operator.scaled_rhs_compact(q, (n,) * dim, h), M @ q)


def _bump(X, dim):
    """smooth bump supported in the ball of radius 0.3 about the centre, and
    its analytic Laplacian"""
    r2 = sum((Xa - 0.5) ** 2 for Xa in X)
    a = 0.09
    s = np.clip(1 - r2 / a, 0, None)
    u = s ** 6
    # u = s^6, s = 1 - r^2/a: grad s = -2 (x - c)/a, Lap s = -2 dim / a
    ds2 = 4 * r2 / a ** 2
    lap = 6 * 5 * s ** 4 * ds2 + 6 * s ** 5 * (-2 * dim / a)
    return u, lap


def _mms_error(n, dim, kappa_fn):
    h = 1.0 / (n - 1)
    X = _grid(n, dim)
    u, lap = _bump(X, dim)
    kap = kappa_fn(X)
    omega = 12.0
    gamma = 2.0
    sigma = kap ** 2 * omega ** 2 * (1 - 1j * gamma / omega)
    f = -lap - sigma * u
    A = operator.helmholtz_compact((n,) * dim, h, kap.ravel(), omega, np.full(n ** dim, gamma))
    rhs = operator.scaled_rhs_compact(f.ravel(), (n,) * dim, h)
    uh = spla.spsolve(A.tocsc(), rhs)
    return np.max(np.abs(uh - u.ravel()))


@pytest.mark.parametrize("dim,sizes", [(2, (33, 65, 129)), (3, (17, 33))])
def test_mms_fourth_order_constant_medium(dim, sizes):
    errs = [_mms_error(n, dim, lambda X: np.ones_like(X[0])) for n in sizes]
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert min(rates) > 3.6, (errs, rates)


def test_mms_variable_medium_at_least_second_order():
    errs = [_mms_error(n, 2, lambda X: 0.8 + 0.2 * np.sin(2 * np.pi * X[0]) * np.cos(np.pi * X[1]))
            for n in (33, 65, 129)]
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert min(rates) > 1.8, (errs, rates)
