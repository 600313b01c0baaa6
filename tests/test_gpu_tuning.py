"""Tuning tools of Section 5.2 on the GPU against the oracle.

- hz_lfa_factors: mu_loc and rho_loc (Definitions 2.1, 2.2) for 2D 5-point
  and compact 9-point, 3D 7-point and compact 19-point constant stencils with
  a complex shift, every patch, linear / cubic transfer symbols, several
  dampings and relaxation counts, equal to the oracle's LFA (numpy
  eigenvalues of Eq. symbolTG) on the same frequency meshes: mu within 1e-12,
  rho within 1e-8 relative (the GPU's rho comes from its own complex QR
  iteration).
- hz_cycle_factor: Eq. cf of the cycle as a stationary solver for A_s u = 0
  from the same seeded initial guess equals the oracle's
  multigrid.convergence_factor within 1e-6 relative, iteration counts +-1.
- minimal_shift / damping_search pick the same candidate as the same loops
  over the oracle's factors.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pairs import medium  # noqa: E402


def _stencil(kind, dim, n=65, alpha=0.3, ppw=10.0):
    from oracle import operator
    h = 1.0 / (n - 1)
    omega = 2 * np.pi / (ppw * h)
    sigma = omega ** 2 * (1 - 0.01j) - 1j * alpha * omega ** 2
    if kind == "5pt":
        return operator.five_point_stencil(h, sigma, dim)
    return operator.compact9_stencil(h, sigma) if dim == 2 else operator.compact19_stencil(h, sigma)


LFA_CASES = [(2, "5pt", p, k) for p in ("jacobi", "element", "plus", "rb", "full")
             for k in (("cubic", "cubic"), ("linear", "cubic"), ("linear", "linear"))]
LFA_CASES += [(2, "compact", p, ("cubic", "cubic")) for p in ("element", "plus", "rb", "full")]
LFA_CASES += [(3, "5pt", p, ("linear", "linear")) for p in ("jacobi", "element", "plus", "rb")]
LFA_CASES += [(3, "compact", p, ("linear", "cubic")) for p in ("element", "rb", "full")]


@pytest.mark.parametrize("nu", [(1, 1), (2, 1)])
@pytest.mark.parametrize("dim,kind,patch,kinds", LFA_CASES,
                         ids=[f"{c[0]}d-{c[1]}-{c[2]}-{c[3][0]}{c[3][1]}" for c in LFA_CASES])
def test_lfa_factors_match_oracle(dim, kind, patch, kinds, nu):
    from oracle import lfa
    from paper_2511_16808_gb300 import hz
    st = _stencil(kind, dim)
    ws = np.array([0.4, 0.7, 0.95, 1.2])
    samples = 32 if dim == 2 else 8
    mu, rho = hz.hz_lfa_factors(dim, st, patch, ws, kinds[0], kinds[1], nu[0], nu[1], samples)
    for i, w in enumerate(ws):
        mu_o = lfa.mu_loc(st, patch, w, samples=samples)
        rho_o = lfa.rho_loc(st, patch, w, kinds[0], kinds[1], samples=samples, nu1=nu[0], nu2=nu[1])
        assert abs(mu[i] - mu_o) <= 1e-12 * max(1.0, mu_o), (w, mu[i], mu_o)
        assert abs(rho[i] - rho_o) <= 1e-8 * max(1.0, rho_o), (w, rho[i], rho_o)


def test_lfa_singular_patch_rejected():
    from paper_2511_16808_gb300 import hz
    st = {(0, 0): 0.0, (1, 0): 1.0, (-1, 0): 1.0, (0, 1): 0.0, (0, -1): 0.0}
    with pytest.raises(hz.HzError):
        hz.hz_lfa_factors(2, st, "jacobi", [0.8])


CF_CASES = [
    dict(dim=2, n=65, levels=4, patch="rb", scheme="leveldep", kind="layered", alpha=0.25),
    dict(dim=2, n=65, levels=3, patch="plus", scheme="cubic", kind="homogeneous", alpha=0.1),
    dict(dim=3, n=17, levels=3, patch="element", scheme="linear", kind="layered", alpha=0.5),
]


def _oracle_cf(c, alpha, u0, damping=None, max_iter=60):
    from oracle import multigrid, solver as osolver
    h, omega, kappa, gamma = medium(c["dim"], c["n"], 0, 0, 10.0, c["kind"])
    pr = osolver.Problem((c["n"],) * c["dim"], h, kappa, omega, gamma, alpha, c["levels"], c["patch"],
                         c["scheme"], damping=damping)
    return multigrid.convergence_factor(pr.hier, u0, np.zeros_like(u0), max_iter=max_iter)


@pytest.mark.parametrize("c", CF_CASES, ids=[f"{c['dim']}d-n{c['n']}-{c['patch']}" for c in CF_CASES])
def test_cycle_factor_matches_oracle(c):
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    from paper_2511_16808_gb300.tuning import cycle_factor
    h, omega, kappa, gamma = medium(c["dim"], c["n"], 0, 0, 10.0, c["kind"])
    s = HelmholtzSolver(c["dim"], [c["n"]] * c["dim"], kappa, omega, gamma, c["alpha"], c["levels"],
                        patch=c["patch"], intergrid=c["scheme"], precision="fp64")
    N = c["n"] ** c["dim"]
    g = np.random.default_rng(1)
    u0 = g.standard_normal(N) + 1j * g.standard_normal(N)
    cf, its = cycle_factor(s, u0=u0, max_iter=60)
    s.close()
    cf_o = _oracle_cf(c, c["alpha"], u0)
    assert abs(cf - cf_o) <= 1e-6 * cf_o, (cf, cf_o)
    assert 0 < its <= 60


def test_minimal_shift_and_damping_search_match_oracle():
    from paper_2511_16808_gb300.tuning import damping_search, minimal_shift
    c = CF_CASES[1]
    h, omega, kappa, gamma = medium(2, 65, 0, 0, 10.0, "homogeneous")
    alphas = [0.0, 0.05, 0.1, 0.2, 0.3]
    a_gpu, table = minimal_shift(2, 65, kappa, omega, gamma, 3, alphas, patch="plus", intergrid="cubic")
    g = np.random.default_rng(1)
    u0 = g.standard_normal(65 * 65) + 1j * g.standard_normal(65 * 65)
    cf_o = [_oracle_cf(c, a, u0) for a in alphas]
    a_o = next(a for a, f in zip(alphas, cf_o) if f < 1)
    assert a_gpu == a_o == 0.2, (table, cf_o)
    for (a, f, _), fo in zip(table, cf_o):
        assert abs(f - fo) <= 1e-6 * fo
    cands = [0.5, 0.7, 0.9, 1.1]
    w_gpu, wt = damping_search(2, 65, kappa, omega, gamma, 0.2, 3, 0, cands, patch="plus", intergrid="cubic")
    from oracle import defaults
    cf_w = [_oracle_cf(c, 0.2, u0, damping=[w, defaults.damping(2, "plus", 1)]) for w in cands]
    assert w_gpu == cands[int(np.argmin(cf_w))], (wt, cf_w)
