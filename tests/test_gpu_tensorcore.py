"""The coarsest solve of a batched V-cycle on the tcgen05 tensor cores.

hz_coarse_solve_batch runs U = A_L^{-1} F (Algorithm 1 step 3) for R
right-hand sides with a chosen variant: 0 is the CUDA-core complex GEMM, s in
1..16 the tensor-core kernel (tf32 with the 3xTF32 split, FP32 accumulation in
tensor memory) with K split over s CTAs per row tile.  Checked here:
- every tensor-core variant against the oracle's coarsest LU solve in FP64
  (the mixed path's 1e-4 of the largest entry, as for the CUDA-core GEMM), and
  against the CUDA-core variant within the worst-case FP32 rounding bound
  of the two sums;
- the split sums are deterministic (two runs bit for bit);
- R = 16, 32, 64, coarsest levels of 289 (2D), 1089 (2D) and 729 (3D) nodes,
  so row tiles and K chunks end ragged;
- variants the context cannot run are refused (FP64 context, R = 8).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [dict(dim=2, n=65, levels=3), dict(dim=2, n=257, levels=4), dict(dim=3, n=17, levels=2)]


def _pair(case, precision="mixed", nrhs_max=64):
    from oracle import solver as osolver
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    from pairs import medium
    dim, n, levels = case["dim"], case["n"], case["levels"]
    h, omega, kappa, gamma = medium(dim, n, 0, 4)
    patch = "rb" if dim == 2 else "element"
    scheme = "leveldep" if dim == 2 else "linear"
    orc = osolver.Problem((n,) * dim, h, kappa, omega, gamma, 0.25, levels, patch, scheme)
    gpu = HelmholtzSolver(dim, [n] * dim, kappa, omega, gamma, 0.25, levels, patch=patch, intergrid=scheme,
                          precision=precision, tol=1e-7, nrhs_max=nrhs_max)
    return orc, gpu


@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("case", CASES, ids=[f"{c['dim']}d-n{c['n']}-L{c['levels']}" for c in CASES])
def test_tensor_core_coarsest_solve(case, R):
    from paper_2511_16808_gb300 import hz
    orc, gpu = _pair(case)
    Lc = orc.hier[-1]
    nc = Lc.A.shape[0]
    assert hz.hz_level_describe(gpu.ctx, len(orc.hier) - 1)["nodes"] == nc
    rng = np.random.default_rng(R + nc)
    F = (rng.standard_normal((nc, R)) + 1j * rng.standard_normal((nc, R))).astype(np.complex64)
    Fd = torch.tensor(F.ravel(), device="cuda")
    ref = Lc.lu.solve(F.astype(np.complex128))
    scale = np.max(np.abs(ref))
    outs = {}
    for v in (0, 1, 2, 4, 8, 16):
        U = torch.empty_like(Fd)
        hz.hz_coarse_solve_batch(gpu.ctx, Fd, U, R, v)
        torch.cuda.synchronize()
        outs[v] = U.cpu().numpy().reshape(nc, R)
        assert np.max(np.abs(outs[v] - ref)) <= 1e-4 * scale, (v, np.max(np.abs(outs[v] - ref)) / scale)
    # against the CUDA-core product of the same FP32 inverse: both sum nc
    # complex terms in FP32 (the tensor-core products with the 3xTF32 split,
    # relative error ~2^-22), so they differ by at most the two rounding-error
    # bounds, 2 * (2 nc) 2^-22 (|Ainv| |F|) elementwise (worst case)
    Ainv = np.linalg.inv(Lc.A.toarray())
    bound = 4 * nc * 2.0 ** -22 * (np.abs(Ainv) @ np.abs(F.astype(np.complex128)))
    for v in (1, 2, 4, 8, 16):
        assert np.all(np.abs(outs[v] - outs[0]) <= bound), v
    U2 = torch.empty_like(Fd)
    hz.hz_coarse_solve_batch(gpu.ctx, Fd, U2, R, 4)
    torch.cuda.synchronize()
    assert np.array_equal(U2.cpu().numpy().reshape(nc, R), outs[4])
    gpu.close()


def test_tensor_core_variant_refused_where_not_supported():
    from paper_2511_16808_gb300 import hz
    orc, gpu = _pair(CASES[0], "mixed")
    nc = orc.hier[-1].A.shape[0]
    f8 = torch.zeros(nc * 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(hz.HzError) as e:
        hz.hz_coarse_solve_batch(gpu.ctx, f8, torch.empty_like(f8), 8, 2)
    assert e.value.status == 1
    hz.hz_coarse_solve_batch(gpu.ctx, f8, torch.empty_like(f8), 8, 0)
    gpu.close()
    orc, gpu = _pair(CASES[0], "fp64", 16)
    f16 = torch.zeros(nc * 16, dtype=torch.complex128, device="cuda")
    with pytest.raises(hz.HzError):
        hz.hz_coarse_solve_batch(gpu.ctx, f16, torch.empty_like(f16), 16, 1)
    gpu.close()


def test_bounded_wait_gives_up_and_device_stays_usable():
    """The spin-wait every bulk copy and MMA of the tensor-core kernel takes,
    on its own: with nothing arriving on its barrier it gives up after the
    poll limit and reports HZ_ERR_TIMEOUT (no hang, no trap); with the arrival
    it succeeds at once; the device then runs the tensor-core product as
    before."""
    from paper_2511_16808_gb300 import hz
    st, timed_out = hz.hz_check_wait_timeout(1000, False)
    assert st == hz.HZ_ERR_TIMEOUT and timed_out
    st, timed_out = hz.hz_check_wait_timeout(1000, True)
    assert st == hz.HZ_OK and not timed_out
    with pytest.raises(hz.HzError):
        hz.hz_check_wait_timeout(0, False)               # poll limit out of range
    orc, gpu = _pair(CASES[0])
    nc = orc.hier[-1].A.shape[0]
    rng = np.random.default_rng(9)
    F = (rng.standard_normal((nc, 16)) + 1j * rng.standard_normal((nc, 16))).astype(np.complex64)
    Fd = torch.tensor(F.ravel(), device="cuda")
    U = torch.empty_like(Fd)
    hz.hz_coarse_solve_batch(gpu.ctx, Fd, U, 16, 2)
    ref = orc.hier[-1].lu.solve(F.astype(np.complex128))
    assert np.max(np.abs(U.cpu().numpy().reshape(nc, 16) - ref)) <= 1e-4 * np.max(np.abs(ref))
    gpu.close()
