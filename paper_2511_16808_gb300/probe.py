"""Short solves of a named workload, for profiler captures: build the
hierarchy, then run a few FGMRES solves capped at a small iteration count, so a
capture sees the solver's kernels with few launches before them.

Usage: python -m paper_2511_16808_gb300.probe --workload config2 [--side 129 --levels 4]
       [--solves 2] [--max-iter 10] [--precision mixed] [--nrhs 1]
(--side/--levels: the workload's generator at a smaller grid.)
"""
from __future__ import annotations

import argparse


def main():
    import numpy as np
    import torch
    import workloads
    from .solver import HelmholtzSolver

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="config2")
    ap.add_argument("--side", type=int, default=0)
    ap.add_argument("--levels", type=int, default=0)
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--max-iter", type=int, default=10)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--nrhs", type=int, default=1)
    a = ap.parse_args()
    if a.side:
        w = workloads.small_variant(a.workload, a.side, a.levels or 4)
    else:
        w = getattr(workloads, a.workload)()
    if isinstance(w, list):
        w = w[len(w) // 2]
    s = HelmholtzSolver(w.dim, [w.n] * w.dim, w.kappa.ravel(), w.omega, w.gamma.ravel(), w.alpha, w.levels,
                        patch=w.patch, intergrid=w.intergrid, precision=a.precision, tol=w.tol,
                        restart=w.restart, max_iter=a.max_iter, patch_coarse=w.patch_coarse, cycle=w.cycle,
                        nrhs_max=a.nrhs)
    if a.nrhs > 1:
        q = torch.tensor(np.ascontiguousarray(w.rhs_block()[:, : a.nrhs]), device="cuda")
        for _ in range(a.solves):
            s.solve_batch(q)
    else:
        q = torch.tensor(w.rhs(0), device="cuda")
        for _ in range(a.solves):
            s.solve(q)
    torch.cuda.synchronize()
    s.close()
    print("probe done")


if __name__ == "__main__":
    main()
