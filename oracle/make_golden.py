"""Write the oracle's full-size reference results (test infrastructure only).

Runs the FP64 oracle (and nothing else) on a workload from `workloads` and
stores, in tests/golden/oracle_<name>.json: the FGMRES iteration count and
true relative residual at the workload's tolerance, the oracle's seconds per
iteration on this host, and at seeded sampled nodes both the solution at the
workload's tolerance (the result a GPU solve of the same algorithm must
reproduce) and the solution of a tighter solve (tol 1e-10, close to the exact
discrete solution), so that the full-size CUDA result can be checked one
sampled output at a time.  For the multi-source, multi-frequency workload
(config4) the same is stored per frequency for the first BATCH_SOURCES
sources.  Usage: python -m oracle.make_golden config2 config4
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import solver  # noqa: E402

SAMPLES = 4096
BATCH_SOURCES = 2
BATCH_SAMPLES = 1024


# scaled-down instances of a config's generator, for configs whose full size is
# beyond the oracle's reach on one host (name -> (config, side, levels))
SMALL = {"config3_129": ("config3", 129, 4)}


def _workload(name):
    if name in SMALL:
        c, n, lv = SMALL[name]
        return workloads.small_variant(c, n, lv)
    return getattr(workloads, name)()


def run(name: str, out_dir: str = os.path.join(ROOT, "tests", "golden")) -> dict:
    w = _workload(name)
    t0 = time.time()
    pr = solver.from_workload(w)
    t_setup = time.time() - t0
    q = w.rhs(0)
    t0 = time.time()
    p, info = pr.solve(q, tol=w.tol, m=w.restart, max_iter=w.max_iter)
    t_solve = time.time() - t0
    p_ref, info_ref = pr.solve(q, tol=1e-10, m=w.restart, max_iter=20 * w.max_iter)
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(w.nodes, size=min(SAMPLES, w.nodes), replace=False))
    rec = {
        "workload": w.name, "nodes": w.nodes, "levels": w.levels, "alpha": w.alpha,
        "patch": w.patch, "patch_coarse": w.patch_coarse or w.patch, "intergrid": w.intergrid,
        "tol": w.tol,
        "iters": info.iters, "relres_true": info.relres_true,
        "iters_tight": info_ref.iters, "relres_tight": info_ref.relres_true,
        "setup_s": t_setup, "solve_s": t_solve, "s_per_iter": t_solve / max(info.iters, 1),
        "p_norm": float(np.linalg.norm(p)), "p_ref_norm": float(np.linalg.norm(p_ref)),
        "err_at_tol": float(np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref)),
        "sample_idx": idx.tolist(),
        "p_ref_re": p_ref[idx].real.tolist(), "p_ref_im": p_ref[idx].imag.tolist(),
        "p_tol_re": p[idx].real.tolist(), "p_tol_im": p[idx].imag.tolist(),
    }
    path = os.path.join(out_dir, f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(rec, f)
    return rec


def run_batch(name: str, out_dir: str = os.path.join(ROOT, "tests", "golden")) -> dict:
    ws = getattr(workloads, name)()
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(ws[0].nodes, size=min(BATCH_SAMPLES, ws[0].nodes), replace=False))
    freqs = []
    for w in ws:
        pr = solver.from_workload(w)
        per = []
        for k in range(BATCH_SOURCES):
            q = w.rhs(k)
            t0 = time.time()
            p, info = pr.solve(q, tol=w.tol, m=w.restart, max_iter=w.max_iter)
            t_solve = time.time() - t0
            p_ref, info_ref = pr.solve(q, tol=1e-10, m=w.restart, max_iter=20 * w.max_iter)
            per.append({"source": k, "node": list(w.sources[k]), "iters": info.iters,
                        "relres_true": info.relres_true, "iters_tight": info_ref.iters,
                        "s_per_iter": t_solve / max(info.iters, 1),
                        "err_at_tol": float(np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref)),
                        "p_ref_re": p_ref[idx].real.tolist(), "p_ref_im": p_ref[idx].imag.tolist(),
                        "p_tol_re": p[idx].real.tolist(), "p_tol_im": p[idx].imag.tolist()})
        freqs.append({"workload": w.name, "omega": w.omega, "ppw": w.meta["ppw"], "sources": per})
    rec = {"workload": name, "nodes": ws[0].nodes, "levels": ws[0].levels, "alpha": ws[0].alpha,
           "patch": ws[0].patch, "intergrid": ws[0].intergrid, "tol": ws[0].tol,
           "nsrc": len(ws[0].sources), "sample_idx": idx.tolist(), "freqs": freqs}
    with open(os.path.join(out_dir, f"oracle_{name}.json"), "w") as f:
        json.dump(rec, f)
    return rec


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["config2"]:
        if nm == "config4":
            r = run_batch(nm)
            for fr in r["freqs"]:
                print(nm, fr["ppw"], [(s["iters"], s["iters_tight"], round(s["s_per_iter"], 3))
                                      for s in fr["sources"]])
            continue
        r = run(nm)
        print(nm, "iters", r["iters"], "tight", r["iters_tight"], "s/iter", round(r["s_per_iter"], 3))
