"""Design-study table of Section 5.2 run on the GPU through the public solver:
Table const2D, FGMRES(5) iteration counts for the 2D homogeneous medium with
4-level W(1,1) cycles, four smoothers (each with its shift) x three intergrid
schemes x three grids, next to the same settings with V(1,1) cycles, with the
solve time of each.

Inputs follow Section 5: kappa = 1, 10 grid points per wavelength, a 20-cell
absorbing layer with no attenuation inside it otherwise, the point source at
the centre, zero initial guess, relative residual below 1e-6.  --stencil
compact runs the paper's compact fourth-order operator (Section 2.1); the
default 5-point one gives other counts (on it the RB patch of the finest
level reduces to damped Jacobi).

Usage: python -m paper_2511_16808_gb300.tables [--sizes 129 257 513] [--cycles W V] [--restart 128]
       [--stencil second|compact]
prints one JSON line per cell.
"""
from __future__ import annotations

import argparse
import json
import time

from .solver import HelmholtzSolver

# Table const2D's smoothers and the shift the paper gives each
SMOOTHERS = (("jacobi", 0.3), ("element", 0.25), ("plus", 0.25), ("rb", 0.18))
INTERGRID = ("cubic", "mixed", "leveldep")


def const2d_cell(n: int, patch: str, alpha: float, intergrid: str, cycle: str, levels: int = 4,
                 tol: float = 1e-6, precision: str = "mixed", repeats: int = 2, restart: int = 5,
                 stencil: str = "second") -> dict:
    import torch
    import workloads
    h = 1.0 / (n - 1)
    omega = workloads.omega_for_ppw(10.0, h, v_min=1.0)
    kappa = workloads.homogeneous_kappa(n, 2, 1.0).ravel()
    gamma = workloads.absorbing_gamma((n, n), omega, 0.0, 20).ravel()
    q = workloads.point_source((n, n), ((n - 1) // 2, (n - 1) // 2), h).ravel()
    s = HelmholtzSolver(2, [n, n], kappa, omega, gamma, alpha, levels, patch=patch, intergrid=intergrid,
                        precision=precision, tol=tol, cycle=cycle, restart=restart, stencil=stencil)
    qd = torch.tensor(q, device="cuda")
    p = torch.empty_like(qd)
    s.solve(qd, p)                                            # warm-up (captures the cycle)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    for _ in range(repeats):
        _, info = s.solve(qd, p)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / repeats
    s.close()
    return {"table": "const2D", "cells": n - 1, "omega": omega, "patch": patch, "alpha": alpha,
            "intergrid": intergrid, "cycle": f"{cycle}(1,1)", "levels": levels, "restart": restart,
            "stencil": stencil,
            "iters": info.iters,
            "converged": bool(info.converged), "relres_true": info.relres_true, "ms_per_solve": ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[129, 257, 513])
    ap.add_argument("--cycles", nargs="+", default=["W", "V"])
    ap.add_argument("--restart", type=int, default=5, help="FGMRES restart length (128: non-restarted here)")
    ap.add_argument("--stencil", default="second", choices=["second", "compact"])
    args = ap.parse_args()
    t0 = time.time()
    for n in args.sizes:
        for patch, alpha in SMOOTHERS:
            for ig in INTERGRID:
                for cyc in args.cycles:
                    print(json.dumps(const2d_cell(n, patch, alpha, ig, cyc, restart=args.restart,
                                                  stencil=args.stencil)), flush=True)
    print(json.dumps({"elapsed_s": time.time() - t0}))


if __name__ == "__main__":
    main()
