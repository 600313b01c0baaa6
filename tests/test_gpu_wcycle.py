"""W-cycles (Section 2.2: step 3 of Algorithm 1 replaced by two cycles on the
next level) on the GPU against the oracle's W-cycle, through the C ABI.

- hz_precond_apply with cycle_visits = 2 equals the oracle's W-cycle within the
  single-RHS V-cycle tolerances (FP64 1e-10, mixed 1e-4 of the largest entry),
  for Vanka and Jacobi coarse levels and nu1 = 0, 1, 2 (the second visit's
  pre-relaxation starts from the first visit's result);
- FGMRES(5) with a W-cycle: iteration count within +-1 of the oracle's, host
  FP64 residual below tol, error against a tight oracle solve within the
  V-cycle parity bounds;
- the batched W-cycle (nrhs = 4) equals the oracle per column;
- a two-level W-cycle equals the V-cycle bit for bit (the coarsest level is
  solved once per visit of its parent).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pairs import check_agreement, make_pair, rel_err  # noqa: E402

CASES = [
    dict(dim=2, n=65, levels=4, patch="rb", scheme="leveldep", layer=8),
    dict(dim=2, n=33, levels=3, patch="element", scheme="cubic"),
    dict(dim=2, n=65, levels=4, patch="jacobi", scheme="linear"),
    dict(dim=3, n=17, levels=3, patch="jacobi", scheme="linear", layer=3, patch_coarse="element"),
]


def _ids(cases):
    return [f"{c['dim']}d-n{c['n']}-L{c['levels']}-{c['patch']}"
            + (f"+{c['patch_coarse']}" if c.get("patch_coarse") else "") + f"-{c['scheme']}" for c in cases]


def _pair(case, precision="fp64", nu=(1, 1), nrhs_max=1):
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    from pairs import medium
    from oracle import solver as osolver
    c = dict(case)
    dim, n, levels = c["dim"], c["n"], c["levels"]
    h, omega, kappa, gamma = medium(dim, n, 0, c.get("layer", 0))
    orc = osolver.Problem((n,) * dim, h, kappa, omega, gamma, 0.25, levels, c["patch"], c["scheme"],
                          patch_coarse=c.get("patch_coarse"), nu1=nu[0], nu2=nu[1], cycle="W")
    gpu = HelmholtzSolver(dim, [n] * dim, kappa, omega, gamma, 0.25, levels, patch=c["patch"],
                          intergrid=c["scheme"], precision=precision, tol=1e-7, nu1=nu[0], nu2=nu[1],
                          patch_coarse=c.get("patch_coarse"), nrhs_max=nrhs_max, cycle="W")
    return orc, gpu


def _rand(shape, seed):
    g = np.random.default_rng(seed)
    v = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    return torch.tensor(v, dtype=torch.complex128, device="cuda"), v


@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (0, 1)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
@pytest.mark.parametrize("case", CASES, ids=_ids(CASES))
def test_wcycle_matches_oracle(case, precision, tol, nu):
    orc, gpu = _pair(case, precision, nu)
    N = orc.A.shape[0]
    r, rn = _rand(N, 5)
    z = gpu.precond(r).cpu().numpy()
    zw = orc.precond(rn)
    assert rel_err(z, zw) < tol
    orc.cycle = "V"
    assert rel_err(zw, orc.precond(rn)) > 1e-3               # the W-cycle differs from the V-cycle
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES[:1] + CASES[3:], ids=_ids(CASES[:1] + CASES[3:]))
def test_wcycle_fgmres(case, precision):
    import workloads
    orc, gpu = _pair(case, precision)
    n, dim = case["n"], case["dim"]
    q = workloads.point_source((n,) * dim, tuple([(n - 1) // 2] * dim), 1.0 / (n - 1)).ravel()
    p_o, info_o = orc.solve(q, tol=1e-7)
    p_ref, _ = orc.solve(q, tol=1e-10)
    p, info = gpu.solve(torch.tensor(q, device="cuda"))
    p = p.cpu().numpy()
    assert info.converged == 1 and abs(info.iters - info_o.iters) <= 1, (info.iters, info_o.iters)
    qh = orc.rhs(q)
    assert np.linalg.norm(qh - orc.A @ p) / np.linalg.norm(qh) < 1e-7
    check_agreement(p, p_o, p_ref, precision, "W")
    gpu.close()


@pytest.mark.parametrize("case", CASES[1:2] + CASES[3:], ids=_ids(CASES[1:2] + CASES[3:]))
def test_batched_wcycle(case):
    orc, gpu = _pair(case, "fp64", nrhs_max=4)
    N = orc.A.shape[0]
    v, vn = _rand((N, 4), 9)
    z = gpu.precond(v).cpu().numpy()
    for r in range(4):
        assert rel_err(z[:, r], orc.precond(vn[:, r])) < 1e-10
    gpu.close()


def test_two_level_w_equals_v():
    case = dict(dim=2, n=33, levels=2, patch="plus", scheme="leveldep")
    orc, gw = _pair(case)
    _, gv = make_pair(2, 33, 2, "plus", "leveldep", alpha=0.25)
    r, _ = _rand(33 * 33, 2)
    assert torch.equal(gw.precond(r), gv.precond(r))
    gw.close()
    gv.close()
