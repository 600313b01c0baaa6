"""CUDA path vs the FP64 oracle, element by element, one test per row of the
hot path, through the C ABI, for the 5-/7-point operator and for the compact
fourth-order stencils (hz_opts.stencil = 1).

Tolerances: the FP64 path runs the same arithmetic in a different order, so
relative differences are rounding-level (<= 1e-11 relative to the largest
entry, allowing for the growth of rounding through a few stencil and
inverse applications).  The mixed path stores the V-cycle in complex FP32
(unit roundoff 6e-8); one V-cycle of a few dozen stencil applications keeps
the relative error below 1e-4 of the largest entry.  FGMRES iteration counts
must agree within +-1 and the converged solution within 1e-6 (FP64) /
1e-5 (mixed) relative L2 of the oracle's solution at the same tolerance; the
error against an oracle solve to 1e-10 is reported beside it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pairs import check_agreement, make_pair, oracle_planes, rel_err  # noqa: E402

CASES_2D = [
    dict(dim=2, n=65, levels=3, patch="rb", scheme="leveldep", layer=8),
    dict(dim=2, n=65, levels=3, patch="plus", scheme="leveldep", layer=8),
    dict(dim=2, n=33, levels=3, patch="element", scheme="cubic"),
    dict(dim=2, n=33, levels=2, patch="full", scheme="mixed"),
    dict(dim=2, n=33, levels=3, patch="jacobi", scheme="linear"),
    dict(dim=2, n=129, levels=4, patch="plus", scheme="leveldep", kind="homogeneous"),
]
CASES_3D = [
    dict(dim=3, n=17, levels=3, patch="element", scheme="linear", layer=3),
    dict(dim=3, n=9, levels=2, patch="plus", scheme="leveldep"),
    dict(dim=3, n=9, levels=2, patch="rb", scheme="cubic"),
    # the heterogeneous 3D smoother choices of Section 5.5: Jacobi on the fine level
    # with element Vanka below it, and plain damped Jacobi with trilinear intergrid
    dict(dim=3, n=17, levels=3, patch="jacobi", scheme="linear", layer=3, patch_coarse="element"),
    dict(dim=3, n=17, levels=4, patch="jacobi", scheme="linear", layer=3),
]
# the compact fourth-order stencils of Section 2.1 as the solved operator
CASES_COMPACT = [
    dict(dim=2, n=65, levels=3, patch="rb", scheme="leveldep", layer=8, stencil="compact"),
    dict(dim=2, n=33, levels=3, patch="element", scheme="cubic", stencil="compact"),
    dict(dim=2, n=129, levels=4, patch="plus", scheme="leveldep", kind="homogeneous", stencil="compact"),
    dict(dim=3, n=17, levels=3, patch="element", scheme="linear", layer=3, stencil="compact"),
]
ALL = CASES_2D + CASES_3D + CASES_COMPACT


def _ids(cases):
    return [f"{c['dim']}d-n{c['n']}-L{c['levels']}-{c['patch']}"
            + (f"+{c['patch_coarse']}" if c.get("patch_coarse") else "") + f"-{c['scheme']}"
            + ("-compact" if c.get("stencil") == "compact" else "") for c in cases]


def case_id(c):
    return _ids([c])[0]


def _pair(case, precision="fp64"):
    c = dict(case)
    return make_pair(c.pop("dim"), c.pop("n"), c.pop("levels"), c.pop("patch"), c.pop("scheme"),
                     precision=precision, **c)


def _rand(N, seed, dtype=torch.complex128):
    g = np.random.default_rng(seed)
    v = g.standard_normal(N) + 1j * g.standard_normal(N)
    return torch.tensor(v, dtype=dtype, device="cuda"), v


@pytest.mark.parametrize("case", ALL, ids=_ids(ALL))
def test_operator_apply(case):
    orc, gpu = _pair(case)
    N = orc.A.shape[0]
    v, vn = _rand(N, 1)
    for shifted, A in ((0, orc.A), (1, orc.A_s)):
        w = gpu.apply(v, shifted=bool(shifted)).cpu().numpy()
        if case.get("stencil") == "compact":
            # up to 27 terms of size |A_pq v_q| summed in another order: FP64
            # rounding bound 32 u (|A| |v|) elementwise
            bound = 32 * 2.0 ** -53 * (abs(A) @ np.abs(vn))
            assert np.all(np.abs(w - A @ vn) <= bound)
        else:
            assert rel_err(w, A @ vn) < 1e-13
    gpu.close()


@pytest.mark.parametrize("case", ALL, ids=_ids(ALL))
def test_galerkin_operators(case):
    from paper_2511_16808_gb300 import hz
    orc, gpu = _pair(case)
    L = hz.hz_level_count(gpu.ctx)
    assert L == len(orc.hier)
    for l in range(L):
        d = hz.hz_level_describe(gpu.ctx, l)
        assert d["n"][: case["dim"]] == orc.hier[l].shape
        got = hz.hz_level_export(gpu.ctx, l, 0)
        ref = oracle_planes(orc.hier[l].A, orc.hier[l].shape, d["stencil"])
        assert rel_err(got, ref) < 1e-12, l
        # every stored oracle entry is covered by the GPU stencil
        assert abs(np.abs(got).sum() - np.abs(orc.hier[l].A.data).sum()) <= 1e-9 * np.abs(got).sum()
    gpu.close()


@pytest.mark.parametrize("case", ALL, ids=_ids(ALL))
def test_vanka_sum(case):
    from paper_2511_16808_gb300 import hz
    orc, gpu = _pair(case)
    for l in range(len(orc.hier) - 1):
        d = hz.hz_level_describe(gpu.ctx, l)
        assert abs(d["damping"] - orc.hier[l].w) == 0.0
        got = hz.hz_level_export(gpu.ctx, l, 1)
        ref = oracle_planes(orc.hier[l].M, orc.hier[l].shape, d["smoother"])
        assert rel_err(got, ref) < 1e-11, l
        assert abs(np.abs(got).sum() - np.abs(orc.hier[l].M.data).sum()) <= 1e-9 * np.abs(got).sum()
    gpu.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
@pytest.mark.parametrize("case", ALL, ids=_ids(ALL))
def test_level_components(case, precision, tol):
    """residual, one sweep, restriction, prolongation, coarsest solve."""
    from paper_2511_16808_gb300 import hz
    from oracle import vanka
    orc, gpu = _pair(case, precision)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    L = len(orc.hier)
    for l in range(L):
        Lv = orc.hier[l]
        N = Lv.A.shape[0]
        u, un = _rand(N, 10 + l, dt)
        f, fn = _rand(N, 20 + l, dt)
        if precision == "mixed":
            un, fn = u.cpu().numpy().astype(np.complex128), f.cpu().numpy().astype(np.complex128)
        if l == L - 1:
            x = torch.empty_like(f)
            hz.hz_coarse_solve(gpu.ctx, f, x)
            ref = Lv.lu.solve(fn)
            assert rel_err(x.cpu().numpy(), ref) < (1e-10 if precision == "fp64" else 1e-4)
            continue
        r = torch.empty_like(u)
        hz.hz_level_residual(gpu.ctx, l, u, f, r)
        assert rel_err(r.cpu().numpy(), fn - Lv.A @ un) < tol
        u2 = u.clone()
        hz.hz_level_smooth(gpu.ctx, l, u2, f)
        assert rel_err(u2.cpu().numpy(), vanka.sweep(Lv.A, Lv.M, Lv.w, un, fn)) < tol * 10
        Nc = orc.hier[l + 1].A.shape[0]
        fc = torch.empty(Nc, dtype=dt, device="cuda")
        hz.hz_level_restrict(gpu.ctx, l, f, fc)
        assert rel_err(fc.cpu().numpy(), Lv.R @ fn) < tol
        ec, ecn = _rand(Nc, 30 + l, dt)
        if precision == "mixed":
            ecn = ec.cpu().numpy().astype(np.complex128)
        u3 = u.clone()
        hz.hz_level_prolong_add(gpu.ctx, l, ec, u3)
        assert rel_err(u3.cpu().numpy(), un + Lv.P @ ecn) < tol
    gpu.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
@pytest.mark.parametrize("case", ALL, ids=_ids(ALL))
def test_vcycle(case, precision, tol):
    orc, gpu = _pair(case, precision)
    N = orc.A.shape[0]
    r, rn = _rand(N, 5)
    z = gpu.precond(r).cpu().numpy()
    assert rel_err(z, orc.precond(rn)) < tol
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ALL, ids=_ids(ALL))
def test_fgmres_solve(case, precision):
    orc, gpu = _pair(case, precision)
    n, dim = case["n"], case["dim"]
    src = tuple([(n - 1) // 2] * dim)
    import workloads
    q = workloads.point_source((n,) * dim, src, 1.0 / (n - 1)).ravel()
    tol = 1e-7
    p_o, info_o = orc.solve(q, tol=tol)
    p_ref, _ = orc.solve(q, tol=1e-10)
    qd = torch.tensor(q, device="cuda")
    p, info = gpu.solve(qd)
    p = p.cpu().numpy()
    assert info.converged == 1 and info.relres_true < tol
    assert abs(info.iters - info_o.iters) <= 1, (info.iters, info_o.iters)
    # independent FP64 check of the residual on the host
    qh = orc.rhs(q)
    assert np.linalg.norm(qh - orc.A @ p) / np.linalg.norm(qh) < tol
    check_agreement(p, p_o, p_ref, precision, case_id(case))
    gpu.close()


def test_solve_host_buffers_match_device():
    case = CASES_2D[0]
    orc, gpu = _pair(case, "mixed")
    n = case["n"]
    import workloads
    q = workloads.point_source((n, n), (n // 2, n // 2), 1.0 / (n - 1)).ravel()
    p_dev, info_d = gpu.solve(torch.tensor(q, device="cuda"))
    p_host = np.zeros_like(q)
    from paper_2511_16808_gb300 import hz
    ok, infos = hz.hz_solve(gpu.ctx, q, p_host)
    assert ok and infos[0].iters == info_d.iters
    assert np.array_equal(p_host, p_dev.cpu().numpy())
    gpu.close()


LONG = [CASES_2D[0], CASES_3D[0]]


@pytest.mark.parametrize("m", [20, 40])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", LONG, ids=_ids(LONG))
def test_fgmres_long_restart(case, m, precision):
    """FGMRES(m) with m > 16: the Gram-Schmidt passes of the later inner steps
    run in chunks of 16 vectors; counts +-1 and solutions as for m = 5."""
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    from pairs import medium
    import workloads
    c = dict(case)
    dim, n = c["dim"], c["n"]
    h, omega, kappa, gamma = medium(dim, n, 0, c.get("layer", 0))
    from oracle import solver as osolver
    orc = osolver.Problem((n,) * dim, h, kappa, omega, gamma, 0.25, c["levels"], c["patch"], c["scheme"])
    gpu = HelmholtzSolver(dim, [n] * dim, kappa, omega, gamma, 0.25, c["levels"], patch=c["patch"],
                          intergrid=c["scheme"], precision=precision, tol=1e-7, restart=m)
    q = workloads.point_source((n,) * dim, tuple([(n - 1) // 2] * dim), h).ravel()
    p_o, info_o = orc.solve(q, tol=1e-7, m=m)
    p_ref, _ = orc.solve(q, tol=1e-10)
    p, info = gpu.solve(torch.tensor(q, device="cuda"))
    p = p.cpu().numpy()
    gpu.close()
    assert info.converged == 1 and abs(info.iters - info_o.iters) <= 1, (info.iters, info_o.iters)
    qh = orc.rhs(q)
    assert np.linalg.norm(qh - orc.A @ p) / np.linalg.norm(qh) < 1e-7
    check_agreement(p, p_o, p_ref, precision, f"{case_id(case)} m={m}")


def test_non_restarted_fgmres_w_cycle():
    """Non-restarted FGMRES (m = 128 > iterations) with 4-level W(1,1) cycles on
    the 2D homogeneous medium of Table const2D: the oracle's count +-1, and no
    more iterations than GMRES(5)."""
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    from oracle import solver as osolver
    import workloads
    n = 129
    h = 1.0 / (n - 1)
    omega = workloads.omega_for_ppw(10.0, h, 1.0)
    kappa = np.ones(n * n)
    gamma = workloads.absorbing_gamma((n, n), omega, 0.0, 20).ravel()
    q = workloads.point_source((n, n), (64, 64), h).ravel()
    orc = osolver.Problem((n, n), h, kappa, omega, gamma, 0.25, 4, "element", "leveldep", cycle="W")
    _, info_o = orc.solve(q, tol=1e-6, m=128)
    its = {}
    for m in (128, 5):
        s = HelmholtzSolver(2, [n, n], kappa, omega, gamma, 0.25, 4, patch="element", intergrid="leveldep",
                            precision="fp64", tol=1e-6, restart=m, cycle="W")
        _, info = s.solve(torch.tensor(q, device="cuda"))
        s.close()
        assert info.converged == 1
        its[m] = info.iters
    assert abs(its[128] - info_o.iters) <= 1 and its[128] < 128, (its, info_o.iters)
    assert its[128] <= its[5]
