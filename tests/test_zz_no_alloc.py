"""The allocation-free sweep, hz_level_smooth_noalloc, against hz_level_smooth.

Some callers must not allocate device memory while they call into the
library: for example a process whose GPU memory is reserved up front by its
own allocator or capped by a fixed budget, where one more cudaMalloc could
fail or fragment that reservation.  hz_level_smooth_noalloc is for them: the
same additive Vanka sweep, with its residual kept in scratch that the
library holds in static device memory instead of a buffer of the context.

The test runs both entry points through the C ABI on the same inputs, twice
in a row with different inputs (the shared scratch keeps the previous call's
contents, which must not show up in the next result), with the tolerances of
the other parity tests, and checks that a level above the stated maximum
size is refused with HZ_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(n, levels, precision):
    import workloads
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    h = 1.0 / (n - 1)
    kappa = workloads.layered_kappa_2d(n, 3)
    omega = workloads.omega_for_ppw(10.0, h, 1.5)
    gamma = workloads.absorbing_gamma(kappa.shape, omega, 0.01, 8)
    return HelmholtzSolver(2, [n, n], kappa.ravel(), omega, gamma.ravel(), 0.1, levels, patch="plus",
                           intergrid="leveldep", precision=precision)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_noalloc_sweep_matches_regular_sweep(precision, tol):
    from paper_2511_16808_gb300 import hz
    s = _solver(65, 3, precision)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    rng = np.random.default_rng(7)
    for level in range(hz.hz_level_count(s.ctx) - 1):
        N = hz.hz_level_describe(s.ctx, level)["nodes"]
        for call in range(2):
            u = torch.tensor(rng.standard_normal(N) + 1j * rng.standard_normal(N), dtype=dt, device="cuda")
            f = torch.tensor(rng.standard_normal(N) + 1j * rng.standard_normal(N), dtype=dt, device="cuda")
            ua, ub = u.clone(), u.clone()
            hz.hz_level_smooth(s.ctx, level, ua, f)
            hz.hz_level_smooth_noalloc(s.ctx, level, ub, f)
            torch.cuda.synchronize()
            a, b = ua.cpu().numpy(), ub.cpu().numpy()
            assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(a)), (level, call)
    s.close()


def test_noalloc_rejects_level_above_maximum():
    from paper_2511_16808_gb300 import hz
    s = _solver(513, 5, "mixed")
    n0 = hz.hz_level_describe(s.ctx, 0)["nodes"]
    assert n0 > hz.NOALLOC_MAX_NODES
    u = torch.zeros(n0, dtype=torch.complex64, device="cuda")
    with pytest.raises(hz.HzError) as e:
        hz.hz_level_smooth_noalloc(s.ctx, 0, u, u.clone())
    assert e.value.status == 1
    assert "at most" in hz.hz_last_error()
    n1 = hz.hz_level_describe(s.ctx, 1)["nodes"]
    u1 = torch.zeros(n1, dtype=torch.complex64, device="cuda")
    hz.hz_level_smooth_noalloc(s.ctx, 1, u1, torch.ones_like(u1))
    torch.cuda.synchronize()
    s.close()
