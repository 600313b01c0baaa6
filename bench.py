#!/usr/bin/env python
"""Benchmark: FGMRES(5) + Vanka-smoothed shifted-Laplacian V(1,1) solves/s.

Workload (default): the 2D layered medium, 1025 x 1025 nodes (h = 1/1024),
seeded (seed 0), 10 points per wavelength at v_min = 1.5, gamma/omega =
0.01, 20-cell absorbing layer + first-order ABC, centre point source,
6-level V(1,1) with RB-patch additive Vanka (level-dependent intergrid,
shift alpha = 0.1), complex-FP32 V-cycle inside FP64 FGMRES(5), tol 1e-6.

One step = one complete solve (zero initial guess to relative residual
1e-6) through the C ABI on device-resident inputs; the hierarchy is set up
once before timing (the paper times the Krylov iterations only).  The
working set per solve (~0.5 GB) exceeds the 129 MB L2, so no flush is
needed between steps.  e2e repeats the step with the source in pinned host
memory and the solution returned to host memory (copies inside the timed
region).  The plain FP64 GPU path is timed beside it, and the FP64 CPU
oracle on a bounded sample of the same solve (cpu_baseline).

The default run also times config 3 (the 3D geophysical medium at 257^3,
the largest single-GPU configuration) as extra keys: its mixed and plain
FP64 solves/s, iterations and V-cycle HBM roofline.

`--probe` runs short solves of a workload for profiler captures (no timing,
no JSON line): the hierarchy is built, then a few FGMRES solves capped at a
small iteration count, so a capture sees the solver's kernels with few
launches before them.

Multi-GPU: independent replicas (one solve stream per rank, no data-path
collective); value = all ranks' solves / max-over-ranks time.
`--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

# The oracle runs on one host core when it is the reference arm: the numerical
# libraries size their thread pools when they are imported, so the limits are
# set before numpy is.
if any(a == "--impl=reference" for a in sys.argv) or any(
        a == "--impl" and i + 1 < len(sys.argv) and sys.argv[i + 1] == "reference" for i, a in enumerate(sys.argv)):
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s @ rel-res 1e-6 (mixed vs plain FP64); Vanka DOF/s; p50/p99 latency"
UNIT = "solves/s"


def replica_throughput(dist, units_local, ms_local, device):
    """Whole-job throughput of independent replicas (one per rank, no data-path
    collective): every rank processed units_local units in ms_local ms; the
    value is all ranks' units over the slowest rank's time.  Returns (value,
    max ms)."""
    if dist is None:
        return units_local / (ms_local / 1e3), ms_local
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return float(u.item()) / (ms_max / 1e3), ms_max


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


# FP64 peak of the GB300 from unit counts and clock: 2 DFMA lanes per SM per
# cycle (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained =
# 304/cycle over 152 SMs) x 2 flops x 2070 MHz = 1.259 TFLOP/s.  Used only
# when the measurement below fails.
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.070e9 / 1e12
_FP64_PEAK = {}


def fp64_peak():
    """(TFLOP/s, note): the FP64 DFMA rate measured on this device by the
    library's chain kernel (hz_measure_peak, best of 5 launches), measured
    once per process before the timed regions; else the derived figure."""
    if not _FP64_PEAK:
        try:
            from paper_2511_16808_gb300 import hz
            t, ms = hz.hz_measure_peak("fp64")
            t32, _ = hz.hz_measure_peak("fp32")
            _FP64_PEAK.update(value=t, note=f"measured: DFMA chain kernel ({ms:.2f} ms launch), "
                                            f"{t:.3f} TFLOP/s FP64, {t32:.1f} TFLOP/s FP32 (FFMA)")
        except Exception as e:  # noqa: BLE001
            _FP64_PEAK.update(value=FP64_PEAK_DERIVED,
                              note=f"derived from DFMA rate x SMs x max clock (measurement failed: {e})")
    return _FP64_PEAK["value"], _FP64_PEAK["note"]


def _traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, if one was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            d = json.load(f)
        return d.get(workload, {}).get(kernel)
    except Exception:  # noqa: BLE001
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi start-up (NVML init) must not overlap the timed work
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.05)
            self.skip = len(self.lines)
        except Exception:  # noqa: BLE001
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        import statistics
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "skip", 0):] or self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_solver(w, precision, stream=None, nrhs_max=1):
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    return HelmholtzSolver(w.dim, [w.n] * w.dim, w.kappa.ravel(), w.omega, w.gamma.ravel(), w.alpha,
                           w.levels, patch=w.patch, intergrid=w.intergrid, precision=precision,
                           tol=w.tol, restart=w.restart, nu1=w.nu1, nu2=w.nu2, max_iter=w.max_iter,
                           patch_coarse=w.patch_coarse, nrhs_max=nrhs_max, stream=stream, cycle=w.cycle)


def _workload(name):
    """(workload, index): config4 yields one workload per frequency; its CPU
    sample runs the middle frequency (10 points per wavelength)."""
    import workloads
    w = getattr(workloads, name)()
    return (w[1], 1) if isinstance(w, list) else (w, None)


def oracle_agreement(name, p):
    """Relative L2 error of the solution p (device or host, full field) at the
    sampled nodes stored by oracle/make_golden.py for workload `name`: against
    the oracle's solution at the same tolerance and against its 1e-10 solve.
    None when no stored oracle result exists for the workload."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if not name or not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    if "p_tol_re" not in g:
        return None
    idx = np.array(g["sample_idx"])
    pv = p.cpu().numpy() if hasattr(p, "cpu") else np.asarray(p)
    pv = pv[idx]
    at_tol = np.array(g["p_tol_re"]) + 1j * np.array(g["p_tol_im"])
    tight = np.array(g["p_ref_re"]) + 1j * np.array(g["p_ref_im"])
    return {"vs_oracle_at_tol": float(np.linalg.norm(pv - at_tol) / np.linalg.norm(at_tol)),
            "vs_oracle_tight": float(np.linalg.norm(pv - tight) / np.linalg.norm(tight)),
            "oracle_iters": g["iters"], "samples": int(len(idx))}


def tune(solver, nrhs, args):
    """Autotune the solver's kernel choices before anything is timed (part of
    set-up, like building the hierarchy); returns the chosen candidates."""
    if args.no_autotune:
        return None
    from paper_2511_16808_gb300 import tuning
    entries, _ = tuning.autotune(solver, nrhs, reps=5, cache=args.tune_cache, log=None)
    return [{"level": e["level"], "knob": e["knob"], "candidate": e["candidate"], "us": round(e["us"], 2),
             "others_us": [round(o["us"], 2) for o in entries
                           if (o["kind"], o["level"]) == (e["kind"], e["level"]) and not o["chosen"]]}
            for e in entries if e["chosen"]]


def time_solves(torch, solver, q, p, steps, stream):
    """Device time (ms) of `steps` consecutive solves with CUDA events on the launching stream."""
    from paper_2511_16808_gb300 import hz
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    infos = []
    for _ in range(steps):
        ok, inf = hz.hz_solve(solver.ctx, q, p, 1, stream)
        infos.append(inf[0])
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end), infos


# Workloads whose oracle setup does not fit a bounded CPU sample: the oracle
# runs the same generator at a smaller side and its time per iteration is
# scaled by the node ratio (the V-cycle and Krylov work are linear in nodes).
CPU_SAMPLE_SMALL = {"config3": (129, 4)}


def cpu_baseline_sample(workload: str, iters: int, ref_iters: float):
    """Run the oracle in a fresh single-threaded process on a bounded sample
    (setup, then `iters` FGMRES iterations of the same solve)."""
    small = CPU_SAMPLE_SMALL.get(workload)
    make = (f"workloads.small_variant({workload!r}, {small[0]}, {small[1]})" if small
            else f"getattr(workloads, {workload!r})()")
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import workloads
from oracle import solver, fgmres
w = {make}
w = w[1] if isinstance(w, list) else w
pr = solver.from_workload(w)
q = pr.rhs(w.rhs(0))
t = time.perf_counter()
x, info = fgmres.fgmres(pr.A, q, pr.precond, m=w.restart, tol=w.tol, max_iter={iters})
dt = time.perf_counter() - t
print(json.dumps({{"s_per_iter": dt / info.iters, "iters": info.iters}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    scale, note = 1.0, ""
    if small:
        import workloads
        full = getattr(workloads, workload)()
        scale = full.nodes / small[0] ** full.dim
        note = (f" (oracle run on the same generator at {small[0]}^{full.dim}, {small[1]} levels; "
                f"time per iteration scaled by the node ratio {scale:.2f})")
    s_per_solve = d["s_per_iter"] * scale * ref_iters
    return {"value": 1.0 / s_per_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{workload}: setup untimed, then {d['iters']} FGMRES iterations of the same "
                      f"solve timed ({d['s_per_iter'] * 1e3:.1f} ms/iteration) and scaled by the "
                      f"{ref_iters:g} iterations a full solve takes" + note}


LFA_SWEEPS = (  # (dim, patch, samples per axis, dampings, transfer kinds, grid side)
    (2, "rb", 256, 64, ("cubic", "cubic"), 513),
    (3, "element", 48, 32, ("linear", "linear"), 129),
)


def _lfa_stencil(dim, n, alpha=0.2, ppw=10.0):
    """Constant 5-/7-point shifted stencil (offset tuple -> value) at 10 ppw."""
    h = 1.0 / (n - 1)
    omega = 2 * np.pi / (ppw * h)
    sigma = omega ** 2 * (1 - 0.01j) - 1j * alpha * omega ** 2
    st = {tuple([0] * dim): 2.0 * dim / h ** 2 - sigma}
    for a in range(dim):
        for sgn in (-1, 1):
            off = [0] * dim
            off[a] = sgn
            st[tuple(off)] = -1.0 / h ** 2
    return st


def run_lfa(args):
    """The LFA damping sweep of Section 5.2 (mu_loc and rho_loc for many
    dampings at once) on the GPU; cpu_baseline: the oracle's LFA on two of the
    dampings of each sweep, scaled per (damping, frequency) evaluation."""
    import torch
    from paper_2511_16808_gb300 import hz
    rank, world, local = _env_rank()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    total_evals, total_s, lines = 0, 0.0, []
    with ClockSampler(local) as clk:
        for dim, patch, samples, nw, kinds, n in LFA_SWEEPS:
            st = _lfa_stencil(dim, n)
            ws = np.linspace(0.3, 1.3, nw)
            for _ in range(args.warmup):
                hz.hz_lfa_factors(dim, st, patch, ws, kinds[0], kinds[1], 1, 1, samples)
            t = time.perf_counter()
            for _ in range(args.steps):
                mu, rho = hz.hz_lfa_factors(dim, st, patch, ws, kinds[0], kinds[1], 1, 1, samples)
            dt = (time.perf_counter() - t) / args.steps
            ev = nw * samples ** dim
            total_evals += ev
            total_s += dt
            lines.append({"dim": dim, "patch": patch, "samples": samples, "dampings": nw, "ms": dt * 1e3,
                          "best_w_rho": float(ws[int(np.nanargmin(rho))]), "rho_min": float(np.nanmin(rho))})
    cpu = None
    if not args.no_cpu_baseline:
        code = f"""
import sys, time, json
import numpy as np
sys.path.insert(0, {ROOT!r})
import bench
from oracle import lfa
t_eval = 0.0
for dim, patch, samples, nw, kinds, n in bench.LFA_SWEEPS:
    st = bench._lfa_stencil(dim, n)
    t = time.perf_counter()
    for w in (0.7, 1.0):
        lfa.mu_loc(st, patch, w, samples=samples)
        lfa.rho_loc(st, patch, w, kinds[0], kinds[1], samples=samples)
    t_eval += (time.perf_counter() - t) / (2 * samples ** dim)
print(json.dumps({{"s_per_eval": t_eval / len(bench.LFA_SWEEPS)}}))
"""
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
        if r.returncode == 0:
            d = json.loads(r.stdout.strip().splitlines()[-1])
            cpu = {"value": 1.0 / d["s_per_eval"], "unit": "evaluations/s", "cores": 1, "kind": "oracle",
                   "sample": "oracle mu_loc + rho_loc for 2 dampings of each sweep (same meshes), "
                             "time per (damping, frequency) evaluation averaged over the sweeps"}
    return {"metric": "LFA (damping, frequency) evaluations/s (mu_loc and rho_loc)", "value": total_evals / total_s,
            "unit": "evaluations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic (constant shifted stencils at 10 ppw, alpha 0.2)",
            "config": {"workload": "lfa-damping-sweeps", "sweeps": lines,
                       "timing": "wall clock around the synchronous call (allocation, launch, read-back)"},
            "clocks": clk.summary(), "cpu_baseline": cpu, "gpu_launches": 3 * args.steps * len(LFA_SWEEPS),
            "roofline": None}


def _with_overrides(w, args):
    """The workload with the smoother / intergrid / depth options of the command
    line (the smoother comparisons of the 3D heterogeneous experiments)."""
    from dataclasses import replace
    kw = {k: v for k, v in (("levels", args.levels), ("patch", args.patch),
                            ("patch_coarse", args.patch_coarse), ("intergrid", args.intergrid))
          if v is not None}
    return replace(w, **kw) if kw else w


def extra_workload(name, args, stream):
    """A second workload timed in the same run (the largest single-GPU
    configuration beside the headline one): mixed solves/s over a few device-
    timed solves, its iterations, the V-cycle's HBM roofline and the plain
    FP64 path's solves/s.  Reported as extra keys, not as the line's value."""
    import torch
    from paper_2511_16808_gb300 import hz as _hz
    w = getattr(__import__("workloads"), name)()
    peak, src = _peaks()
    solver = make_solver(w, "mixed", stream)
    tuned = tune(solver, 1, args)
    q = torch.tensor(w.rhs(0), device="cuda")
    p = torch.empty_like(q)
    solver.solve(q, p)
    steps = max(1, min(args.steps, 3))
    ms, infos = time_solves(torch, solver, q, p, steps, stream)
    _hz.hz_profile_select(solver.ctx, "vcycle")
    solver.solve(q, p)
    _hz.hz_profile_select(solver.ctx, "vcycle")
    solver.solve(q, p)
    torch.cuda.synchronize()
    vprof = _hz.hz_profile_read(solver.ctx)
    _hz.hz_profile_select(solver.ctx, "none")
    solver.close()
    v_gbs = vprof["bytes"] / (vprof["ms"] / 1e3) / 1e9 if vprof["ms"] else None
    out = {"workload": w.name, "nodes": w.nodes, "levels": w.levels, "patch": w.patch,
           "patch_coarse": w.patch_coarse or w.patch, "intergrid": w.intergrid, "alpha": w.alpha,
           "value": steps / (ms / 1e3), "unit": UNIT, "ms_per_solve": ms / steps, "steps": steps,
           "iters": infos[-1].iters, "relres_true": infos[-1].relres_true, "autotune": tuned,
           "vcycle_roofline": {"bound": "hbm", "achieved": v_gbs, "peak": peak, "unit": "GB/s",
                               "frac": v_gbs / peak if v_gbs else None, "peak_source": src,
                               "avg_vcycle_us": vprof["ms"] * 1e3 / max(vprof["launches"], 1)}}
    if not args.no_fp64:
        s64 = make_solver(w, "fp64", stream)
        s64.solve(q, p)
        ms64, inf64 = time_solves(torch, s64, q, p, 1, stream)
        s64.close()
        out["plain_fp64"] = {"value": 1.0 / (ms64 / 1e3), "unit": UNIT, "iters": inf64[-1].iters,
                             "relres_true": inf64[-1].relres_true, "ms_per_solve": ms64}
    return out


def extra_batched(args):
    """The batched workload (config 4) in the same run, as extra keys: its
    solves/s (device-timed), e2e, iterations, the one-at-a-time comparison and
    the rooflines of its batched V-cycle and FP64 passes."""
    import copy
    a = copy.copy(args)
    a.config, a.steps, a.warmup, a.no_cpu_baseline = "config4", max(1, min(args.steps, 2)), 1, True
    d = run_batched(a)
    keep = ("value", "unit", "ms_per_step", "steps", "solves_per_step", "converged", "relres_true_max", "iters",
            "e2e", "one_at_a_time_mixed", "plain_fp64", "roofline", "roofline_second", "vcycle_roofline",
            "autotune", "config")
    return {k: d[k] for k in keep if k in d} if d else None


def run_ours(args):
    import torch
    import workloads

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w0 = getattr(workloads, args.config)()
    w = _with_overrides(w0, args)
    stream = torch.cuda.current_stream()
    if rank == 0:
        fp64_peak()                  # measured before the timed regions
    solver = make_solver(w, "mixed", stream)
    tuned = tune(solver, 1, args)
    q = torch.tensor(w.rhs(0), device="cuda")
    p = torch.empty_like(q)
    for _ in range(args.warmup):
        solver.solve(q, p)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    from paper_2511_16808_gb300 import hz as _hz
    launches0 = _hz.hz_kernel_launches(solver.ctx)
    with ClockSampler(local) as clk:
        ms, infos = time_solves(torch, solver, q, p, args.steps, stream)
        launches = _hz.hz_kernel_launches(solver.ctx) - launches0
        # further timed regions: the two FP64 Gram-Schmidt passes, each bracketed
        # by CUDA events inside the captured restart cycle
        profs, ms_prof = {}, {}
        for cls in ("gs_apply", "gs_update"):
            _hz.hz_profile_select(solver.ctx, cls)
            solver.solve(q, p)                              # re-capture the cycle with the events
            _hz.hz_profile_select(solver.ctx, cls)          # reset the accumulators
            ms_prof[cls], _ = time_solves(torch, solver, q, p, args.steps, stream)
            profs[cls] = _hz.hz_profile_read(solver.ctx)
        _hz.hz_profile_select(solver.ctx, "none")
    value, ms = replica_throughput(dist, args.steps, ms, "cuda")
    if dist:
        dist.barrier()
    iters = infos[-1].iters
    gold = args.config if w is w0 else ""      # stored oracle results are of the stock workloads
    agree = {"mixed": oracle_agreement(gold, p)} if rank == 0 else {}

    # e2e through the C ABI with host buffers (pinned source, host solution)
    from paper_2511_16808_gb300 import hz
    qh = torch.tensor(w.rhs(0)).pin_memory()
    ph = torch.empty_like(qh).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    hz.hz_solve(solver.ctx, qh, ph, 1, stream)          # re-captures the cycle without events
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(e2e_steps):
        hz.hz_solve(solver.ctx, qh, ph, 1, stream)
    t1.record(stream)
    t1.synchronize()
    e2e_ms = t0.elapsed_time(t1)

    # V-cycle phase (HBM roofline) and Vanka DOF/s: one extra solve, not timed
    _hz.hz_profile_select(solver.ctx, "vcycle")
    solver.solve(q, p)
    _hz.hz_profile_select(solver.ctx, "vcycle")
    solver.solve(q, p)
    torch.cuda.synchronize()
    vprof = _hz.hz_profile_read(solver.ctx)
    _hz.hz_profile_select(solver.ctx, "none")
    smoothed = 0
    for l in range(_hz.hz_level_count(solver.ctx) - 1):
        smoothed += _hz.hz_level_describe(solver.ctx, l)["nodes"] * (w.nu1 + w.nu2)

    out = None
    if rank == 0:
        # plain FP64 GPU path on the same workload
        fp64 = None
        if not args.no_fp64:
            s64 = make_solver(w, "fp64", stream)
            s64.solve(q, p)
            ms64, inf64 = time_solves(torch, s64, q, p, max(1, min(args.steps, 2)), stream)
            agree["fp64"] = oracle_agreement(gold, p)
            fp64 = {"value": max(1, min(args.steps, 2)) / (ms64 / 1e3), "unit": UNIT,
                    "iters": inf64[-1].iters, "relres_true": inf64[-1].relres_true,
                    "ms_per_solve": ms64 / max(1, min(args.steps, 2))}
            s64.close()
        vdofs = smoothed * vprof["launches"] / (vprof["ms"] / 1e3) if vprof["ms"] > 0 else None
        cpu = None
        if not args.no_cpu_baseline and w is w0:           # the oracle sample is of the stock workload
            cpu = cpu_baseline_sample(args.config, args.cpu_iters, iters)
        peak, src = _peaks()
        names = {"gs_apply": "k_gs_dots (FP64 operator on z + the cycle's inner products, one pass)",
                 "gs_update": "k_gs_update (FP64 Gram-Schmidt update + norm + cast of the next V-cycle input)"}
        kern = {"gs_apply": "k_gs_dots", "gs_update": "k_gs_update"}

        def roof(cls):
            pr = profs[cls]
            avg_ms = pr["ms"] / max(pr["launches"], 1)
            achieved = pr["flops"] / max(pr["launches"], 1) / (avg_ms / 1e3) / 1e12
            pk, pnote = fp64_peak()
            return {"kernel": names[cls], "bound": "alu", "achieved": achieved, "peak": pk,
                    "unit": "TFLOP/s", "frac": achieved / pk,
                    "traffic": _traffic(kern[cls], w.name), "launches": pr["launches"],
                    "avg_launch_us": avg_ms * 1e3, "share_of_solve": pr["ms"] / ms_prof[cls],
                    "algorithmic_bytes_per_launch": pr["bytes"] / max(pr["launches"], 1),
                    "hbm_achieved_gbs": pr["bytes"] / (pr["ms"] / 1e3) / 1e9 if pr["ms"] else None,
                    "peak_note": pnote,
                    "measured_in": f"extra timed region of {args.steps} solves with events "
                                   f"({ms_prof[cls] / args.steps:.1f} ms/solve)"}
        dom = max(profs, key=lambda k: profs[k]["ms"])
        roofline = roof(dom)
        roofline_other = roof("gs_update" if dom == "gs_apply" else "gs_apply")
        v_gbs = vprof["bytes"] / (vprof["ms"] / 1e3) / 1e9 if vprof["ms"] else None
        vcycle_roofline = {"bound": "hbm", "achieved": v_gbs, "peak": peak, "unit": "GB/s",
                           "frac": v_gbs / peak if v_gbs else None, "peak_source": src,
                           "avg_vcycle_us": vprof["ms"] * 1e3 / max(vprof["launches"], 1)}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 V-cycle / c128 FGMRES",
            "data": "synthetic (seeded layered medium)",
            "config": {"workload": w.name, "nodes": w.nodes, "levels": w.levels, "patch": w.patch,
                       "patch_coarse": w.patch_coarse or w.patch, "intergrid": w.intergrid, "alpha": w.alpha, "tol": w.tol, "restart": w.restart,
                       "omega": w.omega, "layer_cells": w.layer_cells,
                       "l2": "working set per solve > 129 MB L2 (no flush)",
                       "parallelism": f"replicas x{world}"},
            "iters": iters, "relres_true": infos[-1].relres_true,
            "unknowns_vcycles_per_s": value * w.nodes * iters,
            "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": 16 * w.nodes, "d2h_bytes_per_step": 16 * w.nodes},
            "plain_fp64": fp64,
            "clocks": clk.summary(),
            "roofline": roofline,
            "roofline_second": roofline_other,
            "vcycle_roofline": vcycle_roofline,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "peak_source": src,
            "vanka_dof_per_s": vdofs,
            "autotune": tuned,
            "err_vs_oracle": agree,
        }
        if args.config == "config2" and not args.no_extra:
            out["config3"] = extra_workload("config3", args, stream)
            out["config1"] = extra_workload("config1", args, stream)
            if world == 1:                       # the batched run is a one-process run of its own
                out["config4"] = extra_batched(args)
    solver.close()
    if dist:
        dist.destroy_process_group()
    return out


def _profile_class(torch, hz, solvers, run, cls):
    """Bracket every launch of `cls` with events over one `run()`; returns the
    summed {ms, launches, bytes, flops} over all solvers."""
    for sv in solvers:
        hz.hz_profile_select(sv.ctx, cls)
    run()                                   # re-capture the cycles with the events
    for sv in solvers:
        hz.hz_profile_select(sv.ctx, cls)   # reset the accumulators
    run()
    torch.cuda.synchronize()
    tot = {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0}
    for sv in solvers:
        d = hz.hz_profile_read(sv.ctx)
        for k in tot:
            tot[k] += d[k]
        hz.hz_profile_select(sv.ctx, "none")
    return tot


def run_batched(args):
    """Multi-RHS workload: 64 seeded point sources x 3 frequencies on one
    513^2 medium; one step = the 192 solves, one batched hz_solve (64 RHS,
    RHS innermost) per frequency."""
    import torch
    import workloads
    from paper_2511_16808_gb300 import hz

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ws = getattr(workloads, args.config)()
    R = len(ws[0].sources)
    nsolve = R * len(ws)
    stream = torch.cuda.current_stream()
    if rank == 0:
        fp64_peak()                  # measured before the timed regions
    # --streams 1: the frequencies one after another on one stream; else each
    # frequency's batched solve on its own stream, driven by its own host
    # thread, so the three independent solves overlap on the device
    conc = args.streams > 1
    streams = [torch.cuda.Stream() for _ in ws] if conc else [stream] * len(ws)
    solvers = [make_solver(w, "mixed", st, nrhs_max=R) for w, st in zip(ws, streams)]
    tuned = [tune(sv, R, args) for sv in solvers]
    Qs = [torch.tensor(w.rhs_block(), device="cuda") for w in ws]
    Ps = [torch.empty_like(Q) for Q in Qs]
    torch.cuda.synchronize()

    def step(Qsrc=None, Pdst=None, sequential=False):
        """One batched solve per frequency (sources Qsrc[k], solutions Pdst[k];
        device tensors by default, pinned host tensors for the e2e leg)."""
        Qsrc = Qs if Qsrc is None else Qsrc
        Pdst = Ps if Pdst is None else Pdst
        if not conc or sequential:
            out = []
            for sv, Q, P in zip(solvers, Qsrc, Pdst):
                ok, inf = hz.hz_solve(sv.ctx, Q, P, R, stream)
                out.append(inf)
            return out
        import threading
        mark = torch.cuda.Event()
        mark.record(stream)
        out = [None] * len(ws)

        def one(k):
            streams[k].wait_event(mark)
            out[k] = hz.hz_solve(solvers[k].ctx, Qsrc[k], Pdst[k], R, streams[k])[1]
        th = [threading.Thread(target=one, args=(k,)) for k in range(len(ws))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for st in streams:
            stream.wait_stream(st)
        if any(o is None for o in out):
            raise RuntimeError("a concurrent batched solve failed")
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = sum(hz.hz_kernel_launches(sv.ctx) for sv in solvers)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(args.steps):
            infos = step()
        t1.record(stream)
        t1.synchronize()
    ms = t0.elapsed_time(t1)
    launches = sum(hz.hz_kernel_launches(sv.ctx) for sv in solvers) - launches0
    value, ms = replica_throughput(dist, args.steps * nsolve, ms, "cuda")
    if dist:
        dist.barrier()
    iters = [[i.iters for i in inf] for inf in infos]
    conv = all(i.converged for inf in infos for i in inf)
    relres = max(i.relres_true for inf in infos for i in inf)

    # e2e: sources from pinned host memory, solutions back to host memory
    Qh = [Q.cpu().pin_memory() for Q in Qs]
    Ph = [torch.empty_like(Q).pin_memory() for Q in Qh]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(Qh, Ph)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    out = None
    if rank == 0:
        # kernel rooflines with the frequencies one after another: events
        # around a kernel that shares the device with other streams would
        # time the sharing, not the kernel
        run = lambda: step(sequential=True)  # noqa: E731
        prof = _profile_class(torch, hz, solvers, run, "gs_update")
        first = _profile_class(torch, hz, solvers, run, "gs_apply")
        vprof = _profile_class(torch, hz, solvers, run, "vcycle")
        smoothed = 0
        for l in range(hz.hz_level_count(solvers[0].ctx) - 1):
            smoothed += hz.hz_level_describe(solvers[0].ctx, l)["nodes"] * (ws[0].nu1 + ws[0].nu2)
        # V-cycles of all right-hand sides in the profiled step
        nv = sum(sum(it) for it in iters)
        vdofs = smoothed * nv / (vprof["ms"] / 1e3) if vprof["ms"] > 0 else None

        # the same sources one at a time (bounded subset): mixed, and plain FP64
        def one_at_a_time(precision, per_freq):
            tot_ms, n, its = 0.0, 0, []
            for w, Q in zip(ws, Qs):
                sv = make_solver(w, precision, stream)
                q = Q[:, 0].contiguous()
                p = torch.empty_like(q)
                sv.solve(q, p)
                for k in range(per_freq):
                    q = Q[:, k].contiguous()
                    ms1, inf = time_solves(torch, sv, q, p, 1, stream)
                    tot_ms += ms1
                    n += 1
                    its.append(inf[0].iters)
                sv.close()
            return {"value": n / (tot_ms / 1e3), "unit": UNIT, "solves_timed": n,
                    "iters_mean": sum(its) / len(its)}
        single = one_at_a_time("mixed", 4)
        fp64 = None if args.no_fp64 else one_at_a_time("fp64", 2)
        cpu = None
        if not args.no_cpu_baseline:
            it1 = iters[1]
            cpu = cpu_baseline_sample(args.config, args.cpu_iters, sum(it1) / len(it1))
        peak, src = _peaks()
        wname = ws[0].name.rsplit("-ppw", 1)[0] + f"-x{R}"

        def roof(pr, kernel, label):
            avg_ms = pr["ms"] / max(pr["launches"], 1)
            ach = pr["flops"] / max(pr["launches"], 1) / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else None
            pk, pnote = fp64_peak()
            return {"kernel": label, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                    "frac": ach / pk if ach else None, "traffic": _traffic(kernel, wname),
                    "launches": pr["launches"], "avg_launch_us": avg_ms * 1e3, "total_ms": pr["ms"],
                    "hbm_achieved_gbs": pr["bytes"] / (pr["ms"] / 1e3) / 1e9 if pr["ms"] else None,
                    "peak_note": pnote}
        r_upd = roof(prof, "k_gs_update_b",
                     "k_gs_update_b (FP64 Gram-Schmidt update + per-RHS norms + cast of the next V-cycle input)")
        r_dot = roof(first, "k_gs_dots_b", "k_gs_dots_b (FP64 operator on z + the cycle's per-RHS inner products)")
        roofline, first_roof = (r_dot, r_upd) if first["ms"] >= prof["ms"] else (r_upd, r_dot)
        v_gbs = vprof["bytes"] / (vprof["ms"] / 1e3) / 1e9 if vprof["ms"] else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 V-cycle / c128 FGMRES",
            "data": "synthetic (homogeneous medium, seeded sources)",
            "config": {"workload": f"{ws[0].name.rsplit('-ppw', 1)[0]} x {R} sources x ppw "
                                   + "/".join(f"{w.meta['ppw']:g}" for w in ws),
                       "nodes": ws[0].nodes, "nrhs": R, "frequencies": len(ws), "levels": ws[0].levels,
                       "patch": ws[0].patch, "intergrid": ws[0].intergrid, "alpha": ws[0].alpha,
                       "tol": ws[0].tol, "restart": ws[0].restart,
                       "l2": "working set per batched solve > 129 MB L2 (no flush)",
                       "frequency_streams": args.streams if conc else 1,
                       "parallelism": f"replicas x{world}"},
            "solves_per_step": nsolve, "converged": conv, "relres_true_max": relres,
            "iters": {f"ppw{w.meta['ppw']:g}": {"min": min(it), "max": max(it), "mean": sum(it) / len(it)}
                      for w, it in zip(ws, iters)},
            "unknowns_vcycles_per_s": world * args.steps * ws[0].nodes * nv / (ms / 1e3),
            "e2e": {"value": nsolve / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": 16 * ws[0].nodes * nsolve, "d2h_bytes_per_step": 16 * ws[0].nodes * nsolve},
            "one_at_a_time_mixed": single,
            "plain_fp64": fp64,
            "clocks": clk.summary(),
            "roofline": roofline,
            "roofline_second": first_roof,
            "vcycle_roofline": {"bound": "hbm", "achieved": v_gbs, "peak": peak, "unit": "GB/s",
                                "frac": v_gbs / peak if v_gbs else None, "peak_source": src,
                                "avg_vcycle_us": vprof["ms"] * 1e3 / max(vprof["launches"], 1)},
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "peak_source": src,
            "vanka_dof_per_s": vdofs,
            "autotune": tuned[0],
        }
    for sv in solvers:
        sv.close()
    if dist:
        dist.destroy_process_group()
    return out


def _serve_problem(req):
    """Media, source and settings of one serving request (run in a worker process)."""
    w = req.workload()
    return {"dim": w.dim, "n": w.n, "kappa": w.kappa.ravel(), "gamma": w.gamma.ravel(), "omega": w.omega,
            "q": w.rhs(0), "alpha": w.alpha, "levels": w.levels,
            "opts": dict(patch=w.patch, intergrid=w.intergrid, precision="mixed", tol=w.tol, restart=w.restart,
                         max_iter=w.max_iter, patch_coarse=w.patch_coarse)}


def run_serving(args):
    """Serving stream: requests arrive (Poisson, 40/s) with their own medium,
    size, frequency and source; the request server admits them under the HBM
    budget and overlaps their solves.  One step = the whole stream, replayed
    in real time; latency = completion - arrival."""
    import multiprocessing as mp

    import workloads
    rank, world, local = _env_rank()
    if rank != 0:
        return None
    reqs = workloads.config5(n_requests=args.requests, rate=args.rate, problems=args.problems)
    # media are inputs: the first `pregenerate` are made before timing, the
    # rest while the stream runs, `lookahead` requests ahead of the arrivals
    # (the whole stream's media would not fit host memory: a 2049^2 request
    # carries 134 MB, a 193^3 one 230 MB).  Worker processes are started with
    # spawn before this process touches the GPU.
    pool = mp.get_context("spawn").Pool(max(1, min(args.media_workers, os.cpu_count() or 1)))
    n_pre = min(len(reqs), max(args.pregenerate, 1))
    probs = pool.map(_serve_problem, reqs[:n_pre], chunksize=1)
    import numpy as np
    import torch
    from paper_2511_16808_gb300 import hz
    from paper_2511_16808_gb300.serve import Server
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    torch.cuda.set_device(local)

    def submit(srv, pr, precision=None):
        o = dict(pr["opts"])
        if precision:
            o["precision"] = precision
        return srv.submit(pr["dim"], pr["n"], pr["kappa"], pr["omega"], pr["q"], gamma=pr["gamma"],
                          alpha=pr["alpha"], levels=pr["levels"], **o)

    # warm-up: a few small requests through a server (module load, graph code paths)
    small = [pr for pr in probs if pr["n"] <= 257][:max(args.warmup, 1)]
    with Server() as srv:
        for t in [submit(srv, pr) for pr in small]:
            srv.wait(t)
    torch.cuda.synchronize()
    pending = {}                                   # request index -> media being generated
    nxt = n_pre

    def refill(upto):
        nonlocal nxt
        while nxt < len(reqs) and nxt < upto:
            pending[nxt] = pool.apply_async(_serve_problem, (reqs[nxt],))
            nxt += 1

    refill(n_pre + args.lookahead)
    stats_media = {"n": 0, "bytes": 0}
    lag = []                                       # submit time - scheduled arrival
    with ClockSampler(local) as clk, Server(max_active=args.max_active, setup_threads=args.setup_threads,
                                            group_max=args.group_max) as srv:
        t0 = time.perf_counter()
        tickets = []
        for i, rq in enumerate(reqs):
            if i < n_pre:
                pr = probs[i]
            else:
                pr = pending.pop(i).get()
                refill(i + 1 + args.lookahead)
            dt = rq.arrival_s - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(submit(srv, pr))
            lag.append(time.perf_counter() - t0 - rq.arrival_s)
            stats_media["n"] += 1
            stats_media["bytes"] += pr["kappa"].nbytes + pr["gamma"].nbytes + pr["q"].nbytes
        res = [srv.wait(t) for t in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
    pool.close()
    pool.join()
    lag = np.array(lag)
    infos = [d for _, d in res]
    ok = [d for d in infos if d["state"] == "done" and d["status"] == "HZ_OK"]
    lat = np.array([d["t_done"] - d["t_submit"] for d in ok])
    qd = np.array([d["t_admit"] - d["t_submit"] for d in ok])
    setup = np.array([d["t_start"] - d["t_admit"] for d in ok])
    solve = np.array([d["t_done"] - d["t_start"] for d in ok])
    span = max(d["t_done"] for d in infos) - min(d["t_submit"] for d in infos)
    value = len(ok) / span

    # one at a time on the same GPU (setup + solve, sequential), first K requests
    def one_at_a_time(precision, k):
        t = time.perf_counter()
        its = []
        for pr in probs[:k]:
            o = dict(pr["opts"], precision=precision)
            s = HelmholtzSolver(pr["dim"], [pr["n"]] * pr["dim"], pr["kappa"], pr["omega"], pr["gamma"],
                                pr["alpha"], pr["levels"], **o)
            p, info = s.solve(pr["q"], np.zeros_like(pr["q"]))
            its.append(info.iters)
            s.close()
        torch.cuda.synchronize()
        return {"value": k / (time.perf_counter() - t), "unit": UNIT, "requests": k,
                "iters_mean": float(np.mean(its))}
    k = min(args.one_at_a_time, len(probs))
    k_mixed = min(args.one_at_a_time_mixed, len(probs))
    seq_mixed = one_at_a_time("mixed", k_mixed)             # the stream's first requests, one at a time
    seq_fp64 = one_at_a_time("fp64", k)
    served_k = len([d for d in infos[:k] if d["state"] == "done"]) / max(
        1e-9, max(d["t_done"] for d in infos[:k]) - min(d["t_submit"] for d in infos[:k]))
    mix = {}
    for rq in reqs:
        key = f"{rq.dim}d-{rq.n}"
        mix[key] = mix.get(key, 0) + 1
    # every request's kappa, gamma (FP64) and source (c128) go up, its solution (c128) comes back
    nodes = sum(rq.n ** rq.dim for rq in reqs)
    h2d = nodes * (8 + 8 + 16)
    d2h = nodes * 16
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None  # noqa: E731
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": len(small),
        "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 V-cycle / c128 FGMRES", "data": "synthetic (seeded media per request)",
        "config": {"workload": f"serving stream: {len(reqs)} requests, Poisson {args.rate:g}/s, "
                               "2D sides 257-2049 / 3D sides 65-193, 8-12 points per wavelength",
                   "requests": len(reqs), "rate_per_s": args.rate, "mix": mix, "max_active": st["max_active"],
                   "setup_threads": args.setup_threads, "media_workers": args.media_workers,
                   "problems": args.problems or "one per request", "group_max": args.group_max,
                   "hbm_budget_bytes": st["budget"], "tol": 1e-6,
                   "l2": "each request's working set > 129 MB L2 except the smallest; no flush",
                   "parallelism": "1 GPU, requests overlapped on streams"},
        "served": len(ok), "failed": st["failed"],
        "groups": {"solves": st["groups"], "requests": st["grouped"],
                   "note": "multi-RHS solves that served several requests of one problem together"},
        "not_ok": [{"rid": rq.rid, "dim": rq.dim, "n": rq.n, "medium": rq.generator, "ppw": round(rq.ppw, 2),
                    "status": d["status"], "iters": d["iters"], "relres_true": d["relres_true"]}
                   for rq, d in zip(reqs, infos) if not (d["state"] == "done" and d["status"] == "HZ_OK")],
        "latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "mean": float(lat.mean()) if len(lat) else None},
        "queue_delay_s": {"p50": pct(qd, 50), "p99": pct(qd, 99)},
        "setup_s": {"p50": pct(setup, 50), "p99": pct(setup, 99)},
        "solve_s": {"p50": pct(solve, 50), "p99": pct(solve, 99)},
        "offered_span_s": reqs[-1].arrival_s, "wall_s": wall,
        "media": {"pregenerated": n_pre, "streamed": len(reqs) - n_pre, "lookahead": args.lookahead,
                  "host_bytes_submitted": stats_media["bytes"],
                  "submit_lag_s": {"p50": pct(lag, 50), "p99": pct(lag, 99), "max": float(lag.max())},
                  "note": "submit lag = submit time - scheduled Poisson arrival (media generation "
                          "running behind the arrivals shows here; latency counts from submit)"},
        "peak_hbm_bytes": st["peak_bytes"],
        "one_at_a_time_mixed": seq_mixed, "plain_fp64": seq_fp64,
        "served_vs_one_at_a_time": value / seq_mixed["value"],
        "one_at_a_time_note": "setup + solve per request, sequential, on the stream's first requests "
                              "(mixed: --one-at-a-time-mixed, plain FP64: --one-at-a-time)",
        "served_first_k": {"value": served_k, "unit": UNIT, "requests": k,
                           "note": "first k requests of the stream, served (arrival to completion)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "requests enter and leave through host buffers"},
        "clocks": clk.summary(),
        "roofline": None, "cpu_baseline": None,
        "gpu_launches": st["kernel_launches"],
    }


def run_reference(args):
    rank, world, local = _env_rank()
    if rank != 0:
        return None
    import workloads
    from oracle import fgmres, solver
    w, fi = _workload(args.config)
    gold = os.path.join(ROOT, "tests", "golden", f"oracle_{args.config}.json")
    with open(gold) as f:
        g = json.load(f)
    if fi is None:
        ref_iters = g["iters"]
    else:
        its = [s["iters"] for s in g["freqs"][fi]["sources"]]
        ref_iters = sum(its) / len(its)
    pr = solver.from_workload(w)
    q = pr.rhs(w.rhs(0))
    per_step = args.ref_iters_per_step
    times = []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        fgmres.fgmres(pr.A, q, pr.precond, m=w.restart, tol=w.tol, max_iter=per_step)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    s_per_iter = sum(times) / (len(times) * per_step)
    value = 1.0 / (s_per_iter * ref_iters)
    sample = (f"{w.name}: each step = {per_step} FGMRES iterations of the oracle solve "
              f"(setup untimed); solves/s scaled by the {ref_iters:g} iterations of a full oracle solve")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * s_per_iter * per_step,
            "step": f"{per_step} FGMRES iterations of the oracle's solve of the workload",
            "extrapolated_from_iters": per_step * len(times),
            "ms_per_solve_extrapolated": 1e3 * s_per_iter * ref_iters,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic (seeded layered medium)",
            "config": {"workload": w.name, "nodes": w.nodes, "levels": w.levels},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_probe(args):
    """Short solves of a workload for profiler captures (see the module
    docstring); --side/--levels select the workload's generator at a smaller
    grid."""
    import torch
    import workloads
    torch.cuda.set_device(0)
    if args.side:
        w = workloads.small_variant(args.config, args.side, args.levels or 4)
    else:
        w = _with_overrides(getattr(workloads, args.config)(), args)
    if isinstance(w, list):
        w = w[len(w) // 2]
    from dataclasses import replace
    w = replace(w, max_iter=args.max_iter)
    s = make_solver(w, args.precision, nrhs_max=args.nrhs)
    if args.nrhs > 1:
        q = torch.tensor(np.ascontiguousarray(w.rhs_block()[:, : args.nrhs]), device="cuda")
        for _ in range(args.solves):
            s.solve_batch(q)
    else:
        q = torch.tensor(w.rhs(0), device="cuda")
        for _ in range(args.solves):
            s.solve(q)
    torch.cuda.synchronize()
    s.close()
    print("probe done", file=sys.stderr)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="config2")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the fixed kernel-choice rules")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of kernel choices: read when it holds the workload's level shapes, else written "
                         "(a profiler run then replays the choices of the plain run)")
    ap.add_argument("--no-extra", action="store_true", help="skip the second (3D) workload of the default run")
    ap.add_argument("--cpu-iters", type=int, default=25)
    ap.add_argument("--ref-iters-per-step", type=int, default=5)
    ap.add_argument("--streams", type=int, default=3,
                    help="config4: 1 = frequencies one after another; else one stream and host thread each")
    ap.add_argument("--requests", type=int, default=2000, help="config5: requests in the stream")
    ap.add_argument("--rate", type=float, default=40.0, help="config5: Poisson arrival rate per second")
    ap.add_argument("--max-active", type=int, default=32, help="config5: requests admitted at once")
    ap.add_argument("--one-at-a-time", type=int, default=24,
                    help="config5: requests timed one at a time on the plain FP64 path")
    ap.add_argument("--setup-threads", type=int, default=2, help="config5: hierarchies built concurrently")
    ap.add_argument("--pregenerate", type=int, default=200, help="config5: media generated before timing")
    ap.add_argument("--lookahead", type=int, default=48, help="config5: media generated ahead of the arrivals")
    ap.add_argument("--media-workers", type=int, default=16, help="config5: processes generating media")
    ap.add_argument("--problems", type=int, default=0,
                    help="config5: requests drawn from this many problems (sources differ); 0 = one per request")
    ap.add_argument("--group-max", type=int, default=8,
                    help="config5: queued requests of one problem solved together, at most (0 = alone)")
    ap.add_argument("--one-at-a-time-mixed", type=int, default=200,
                    help="config5: requests re-run one at a time (mixed) for the comparison")
    ap.add_argument("--levels", type=int, default=None, help="override the workload's cycle depth")
    ap.add_argument("--patch", default=None, help="override the fine-level Vanka patch")
    ap.add_argument("--patch-coarse", default=None, help="patch on the coarse levels (default: the fine one)")
    ap.add_argument("--intergrid", default=None, help="override the intergrid scheme")
    ap.add_argument("--probe", action="store_true", help="short solves for profiler captures (no JSON line)")
    ap.add_argument("--side", type=int, default=0, help="--probe: the workload's generator at this grid side")
    ap.add_argument("--solves", type=int, default=2, help="--probe: solves to run")
    ap.add_argument("--max-iter", type=int, default=10, help="--probe: FGMRES iterations per solve")
    ap.add_argument("--precision", default="mixed", help="--probe: mixed or fp64")
    ap.add_argument("--nrhs", type=int, default=1, help="--probe: right-hand sides per solve")
    args = ap.parse_args()
    if args.probe:
        run_probe(args)
        return
    if args.impl == "reference":
        out = run_reference(args)
    elif args.config == "config4":
        out = run_batched(args)
    elif args.config == "config5":
        out = run_serving(args)
    elif args.config == "lfa":
        out = run_lfa(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
