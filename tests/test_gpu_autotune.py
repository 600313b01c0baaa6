"""The kernel-choice autotuner (hz_autotune / hz_tune_set, tuning.autotune).

- Every knob of every level gets timed candidates and exactly one chosen one;
  the kinds present are the ones the context can use (register budget and
  fused tile passes for one right-hand side; RHS pack and the tensor-core
  coarsest product for 16).
- Whatever is chosen, and every other candidate forced with hz_tune_set, the
  solve still agrees with the oracle: iterations +-1 and the solution within
  1e-5 (mixed) of the oracle's at the same tolerance.
- The JSON cache: a second context of the same level shapes takes the stored
  choices instead of timing again.
- hz_tune_set refuses knobs that do not apply.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pairs import check_agreement, make_pair  # noqa: E402


def _problem():
    import workloads
    n = 129
    q = workloads.point_source((n, n), (n // 2, n // 2), 1.0 / (n - 1)).ravel()
    return n, q


def _solve_and_check(orc, gpu, q, tol=1e-7):
    p_o, info_o = orc.solve(q, tol=tol)
    p, info = gpu.solve(torch.tensor(q, device="cuda"))
    assert info.converged == 1 and abs(info.iters - info_o.iters) <= 1, (info.iters, info_o.iters)
    check_agreement(p.cpu().numpy(), p_o, None, "mixed", "autotuned")


def test_autotune_single_rhs_choices_match_oracle(tmp_path):
    from paper_2511_16808_gb300 import hz, tuning
    n, q = _problem()
    orc, gpu = make_pair(2, n, 4, "plus", "leveldep", precision="mixed", layer=8)
    cache = str(tmp_path / "tune.json")
    entries, cached = tuning.autotune(gpu, 1, reps=3, cache=cache, log=None)
    assert not cached
    levels = hz.hz_level_count(gpu.ctx)
    kinds = {(e["kind"], e["level"]) for e in entries}
    for l in range(levels - 1):
        assert (2, l) in kinds
    assert any(k == 3 for k, _ in kinds)              # the coarse 2D levels have the fused-pass knob
    for key in kinds:
        assert sum(e["chosen"] for e in entries if (e["kind"], e["level"]) == key) == 1
        assert all(e["us"] > 0 for e in entries if (e["kind"], e["level"]) == key)
    _solve_and_check(orc, gpu, q)
    # every candidate forced in turn still solves to the oracle's answer
    for kind, level in sorted(kinds):
        cands = [e["candidate"] for e in entries if (e["kind"], e["level"]) == (kind, level)]
        for cnd in cands:
            hz.hz_tune_set(gpu.ctx, kind, level, 1, cnd)
            _solve_and_check(orc, gpu, q)
    gpu.close()
    # same level shapes: the cache supplies the choices
    orc2, gpu2 = make_pair(2, n, 4, "plus", "leveldep", precision="mixed", layer=8, seed=1)
    entries2, cached2 = tuning.autotune(gpu2, 1, reps=3, cache=cache, log=None)
    assert cached2 and entries2 == entries
    _solve_and_check(orc2, gpu2, q)
    gpu2.close()


def test_autotune_batched_includes_tensor_core_product():
    from paper_2511_16808_gb300 import hz
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    from pairs import medium
    from oracle import solver as osolver
    import workloads
    n, R = 65, 16
    h, omega, kappa, gamma = medium(2, n, 0, 8)
    orc = osolver.Problem((n, n), h, kappa, omega, gamma, 0.25, 3, "rb", "leveldep")
    gpu = HelmholtzSolver(2, [n, n], kappa, omega, gamma, 0.25, 3, patch="rb", intergrid="leveldep",
                          precision="mixed", tol=1e-7, nrhs_max=R)
    entries = hz.hz_autotune(gpu.ctx, R, 3)
    kinds = {e["kind"] for e in entries}
    assert 0 in kinds and 1 in kinds
    coarse = [e for e in entries if e["kind"] == 0]
    assert sorted(e["candidate"] for e in coarse) == [0, 1, 2, 4, 8, 16]
    rng = np.random.default_rng(4)
    nodes = [tuple(int(v) for v in rng.integers(2, n - 2, size=2)) for _ in range(R)]
    Q = np.stack([workloads.point_source((n, n), nd, h).ravel() for nd in nodes], axis=1)
    for cand in (0, 2):
        hz.hz_tune_set(gpu.ctx, 0, hz.hz_level_count(gpu.ctx) - 1, R, cand)
        P, infos = gpu.solve_batch(torch.tensor(Q, device="cuda"))
        P = P.cpu().numpy()
        for r in (0, R - 1):
            p_o, info_o = orc.solve(Q[:, r].copy(), tol=1e-7)
            assert infos[r].converged == 1 and abs(infos[r].iters - info_o.iters) <= 1
            check_agreement(P[:, r], p_o, None, "mixed", f"rhs {r} coarse variant {cand}")
    gpu.close()


def test_tune_set_refuses_what_does_not_apply():
    from paper_2511_16808_gb300 import hz
    orc, gpu = make_pair(2, 65, 3, "rb", "leveldep", precision="mixed")
    with pytest.raises(hz.HzError):
        hz.hz_tune_set(gpu.ctx, 0, 0, 1, 0)          # kind 0 belongs to the coarsest level
    with pytest.raises(hz.HzError):
        hz.hz_tune_set(gpu.ctx, 2, 0, 1, 3)          # no such register budget
    with pytest.raises(hz.HzError):
        hz.hz_tune_set(gpu.ctx, 0, 2, 16, 4)         # no tensor-core product without a batch
    gpu.close()
