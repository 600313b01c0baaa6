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
the other parity tests, for a plus patch and an RB patch in 2D and an element
patch in 3D.  It checks that, after a first call, further calls change
neither the library's count of device allocations nor the bytes in use in
the device's stream-ordered pool, and that a level above the stated maximum
size is refused with HZ_ERR_INVALID_ARG.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(2, 65, 3, "plus"), (2, 65, 3, "rb"), (3, 17, 3, "element")]


def _solver(dim, n, levels, patch, precision):
    import workloads
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    h = 1.0 / (n - 1)
    kappa = workloads.layered_kappa_2d(n, 3) if dim == 2 else workloads.geophysical_kappa_3d(n, 3)
    omega = workloads.omega_for_ppw(10.0, h, 1.5)
    gamma = workloads.absorbing_gamma(kappa.shape, omega, 0.01, 8 if dim == 2 else 3)
    return HelmholtzSolver(dim, [n] * dim, kappa.ravel(), omega, gamma.ravel(), 0.1 if dim == 2 else 0.5, levels,
                           patch=patch, intergrid="leveldep" if dim == 2 else "linear", precision=precision)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
@pytest.mark.parametrize("dim,n,levels,patch", CASES, ids=[f"{c[0]}d-{c[3]}" for c in CASES])
def test_noalloc_sweep_matches_regular_sweep(dim, n, levels, patch, precision, tol):
    from paper_2511_16808_gb300 import hz
    s = _solver(dim, n, levels, patch, precision)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    rng = np.random.default_rng(7)
    dev = torch.cuda.current_device()
    for level in range(hz.hz_level_count(s.ctx) - 1):
        N = hz.hz_level_describe(s.ctx, level)["nodes"]
        for call in range(2):
            u = torch.tensor(rng.standard_normal(N) + 1j * rng.standard_normal(N), dtype=dt, device="cuda")
            f = torch.tensor(rng.standard_normal(N) + 1j * rng.standard_normal(N), dtype=dt, device="cuda")
            ua, ub = u.clone(), u.clone()
            hz.hz_level_smooth(s.ctx, level, ua, f)
            torch.cuda.synchronize()
            before = hz.hz_memory_stats(dev)
            hz.hz_level_smooth_noalloc(s.ctx, level, ub, f)
            torch.cuda.synchronize()
            after = hz.hz_memory_stats(dev)
            a, b = ua.cpu().numpy(), ub.cpu().numpy()
            assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(a)), (level, call)
            # the allocation-free call allocated nothing, by the library's own
            # count and by the device pool's bytes in use
            assert after == before, (level, call, before, after)
    s.close()


def test_noalloc_rejects_level_above_maximum():
    from paper_2511_16808_gb300 import hz
    s = _solver(2, 513, 5, "plus", "mixed")
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
