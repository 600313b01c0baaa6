"""Parameter searches of Section 5.2 on the GPU, through the C ABI.

- lfa_damping: mu_loc and rho_loc (Definitions 2.1, 2.2) of additive Vanka for
  a constant stencil over a grid of damping values in one batched LFA sweep
  (hz_lfa_factors); the damping minimising rho_loc (or mu_loc).
- cycle_factor: the convergence factor of Eq. cf of a set-up hierarchy's cycle
  used as a stationary solver (hz_cycle_factor).
- minimal_shift: the smallest shift alpha in a candidate list whose cycle
  converges (c_f < 1) on a small grid, the procedure Section 5.2 describes for
  choosing each smoother's shift.
- damping_search: the per-level exhaustive search of Section 5.2: for level l,
  the damping giving the smallest c_f with the finer levels' dampings fixed.

Every factor is computed by the library's kernels; this module only loops over
the candidates.  Zero right-hand side and a seeded random initial guess, as in
Section 5.1.
"""
from __future__ import annotations

import numpy as np

from . import hz
from .solver import HelmholtzSolver


def lfa_damping(dim, stencil, patch, ws, rk="cubic", pk="cubic", nu1=1, nu2=1, samples=128, by="rho"):
    """(best damping, mu[], rho[]) over the candidate dampings `ws`."""
    ws = np.asarray(ws, dtype=np.float64)
    mu, rho = hz.hz_lfa_factors(dim, stencil, patch, ws, rk, pk, nu1, nu2, samples)
    crit = rho if by == "rho" else mu
    return float(ws[int(np.nanargmin(crit))]), mu, rho


def cycle_factor(solver: HelmholtzSolver, seed: int = 1, warmup: int = 5, target: float = 1e-9,
                 max_iter: int = 300, u0=None):
    """(c_f, iterations) for the solver's cycle on A_s u = 0 from a seeded
    random (or the given) initial guess."""
    import torch
    N = solver.nodes
    if u0 is None:
        g = np.random.default_rng(seed)
        u0 = g.standard_normal(N) + 1j * g.standard_normal(N)
    u = torch.tensor(np.asarray(u0, dtype=np.complex128), device="cuda")
    f = torch.zeros_like(u)
    return hz.hz_cycle_factor(solver.ctx, f, u, warmup, target, max_iter, solver.stream)


def _factor_for(dim, n, kappa, omega, gamma, alpha, levels, seed, cf_max_iter, **opts):
    s = HelmholtzSolver(dim, [n] * dim, kappa, omega, gamma, alpha, levels, precision="fp64", **opts)
    try:
        return cycle_factor(s, seed=seed, max_iter=cf_max_iter)
    finally:
        s.close()


def minimal_shift(dim, n, kappa, omega, gamma, levels, alphas, seed=1, cf_max_iter=60, **opts):
    """(smallest alpha with c_f < 1 or None, [(alpha, c_f, iterations)]),
    trying the candidates in increasing order and stopping at the first one
    that converges.  cf_max_iter bounds the iterations of each factor (a
    divergent cycle's residual grows geometrically)."""
    table = []
    for a in sorted(alphas):
        cf, its = _factor_for(dim, n, kappa, omega, gamma, a, levels, seed, cf_max_iter, **opts)
        table.append((a, cf, its))
        if cf < 1.0:
            return a, table
    return None, table


def damping_search(dim, n, kappa, omega, gamma, alpha, levels, level, candidates, fixed=(), seed=1,
                   patch="rb", patch_coarse=None, cf_max_iter=60, **opts):
    """(best damping for `level`, [(w, c_f)]): dampings of the finer levels
    from `fixed`, the coarser ones from the paper's table."""
    from .solver import make_opts
    base = make_opts(dim, levels, patch=patch, patch_coarse=patch_coarse)
    table = []
    for w in candidates:
        damp = [base.damping[l] for l in range(levels)]
        damp[: len(fixed)] = list(fixed)
        damp[level] = w
        cf, _ = _factor_for(dim, n, kappa, omega, gamma, alpha, levels, seed, cf_max_iter, patch=patch,
                            patch_coarse=patch_coarse, damping=damp, **opts)
        table.append((float(w), cf))
    best = min(table, key=lambda t: t[1])
    return best[0], table


# ---- kernel-choice autotuning (no counterpart in the paper) ----------------

def tune_key(solver: HelmholtzSolver, nrhs: int) -> str:
    """Cache key of a context's tunable shape: device name, V-cycle precision,
    batch width, and per level the grid, operator and smoother stencil sizes
    and patch (what the kernel choices depend on; not the medium)."""
    import json
    import torch
    info = hz.hz_context_info(solver.ctx)
    levels = []
    for l in range(hz.hz_level_count(solver.ctx)):
        d = hz.hz_level_describe(solver.ctx, l)
        levels.append([list(d["n"]), len(d["stencil"]), len(d["smoother"]), d["patch"], d["is_coarsest"]])
    return json.dumps({"device": torch.cuda.get_device_name(info["device"]), "precision": info["precision"],
                       "nrhs": nrhs, "levels": levels}, sort_keys=True)


def autotune(solver: HelmholtzSolver, nrhs: int = 1, reps: int = 10, cache: str | None = None, log=print):
    """Kernel choices for `solver` at batch width nrhs: taken from the JSON
    cache file when it holds this shape (applied with hz_tune_set), else timed
    by hz_autotune, logged candidate by candidate and stored in the cache.
    Returns (entries, from_cache)."""
    import json
    import os
    key = tune_key(solver, nrhs)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        entries = table[key]
        for e in entries:
            if e["chosen"]:
                hz.hz_tune_set(solver.ctx, e["kind"], e["level"], e["nrhs"], e["candidate"])
        return entries, True
    entries = hz.hz_autotune(solver.ctx, nrhs, reps)
    if log:
        for e in entries:
            log(f"autotune level {e['level']} {e['knob']:>17} candidate {e['candidate']}: "
                f"{e['us']:9.2f} us{'  <- chosen' if e['chosen'] else ''}")
    if cache:
        table[key] = entries
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return entries, False
