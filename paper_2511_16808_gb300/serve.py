"""Serving front end over the C ABI's request server (hz_server_*): submits
whole problems (medium, frequency, shift, solver options, one source), holds
each request's host solution buffer until it has finished, and reports the
server's timestamps.  Scheduling, setup and the solves run in libhz's own
threads and kernels; nothing here computes."""
from __future__ import annotations

import numpy as np

import time

from . import hz
from .solver import JsonLines, make_opts


class Server:
    """hbm_budget: device bytes the admitted requests may hold (0: 80% of free
    memory); max_active: requests set up or solving at once (0: 32);
    setup_threads: hierarchies built concurrently (0: 2); group_max: requests
    of the same problem (only the source differs) waiting together are solved
    together as one multi-RHS solve of up to this many right-hand sides (0:
    every request alone); log: a path or text file receiving one JSON line per
    finished request (latency, queue delay, setup and solve spans, iterations,
    bytes, group size) and one with the server's counters when it closes."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 0, device: int = -1, setup_threads: int = 0,
                 log=None, group_max: int = 0):
        self.srv = hz.hz_server_create(hbm_budget, max_active, device, setup_threads, group_max)
        self._keep = {}
        self.log = JsonLines(log) if log is not None else None

    def submit(self, dim, n, kappa, omega, q, gamma=None, alpha=0.25, levels=4, gamma0=0.0, **solver_opts):
        """kappa, gamma, q: host arrays of n^dim values (float64, float64,
        complex128); solver_opts as for HelmholtzSolver.  Returns the ticket."""
        n = list(n) if hasattr(n, "__len__") else [n] * dim
        nodes = int(np.prod(n[:dim]))
        k = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64).reshape(-1))
        g = None if gamma is None else np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(-1))
        qq = np.ascontiguousarray(np.asarray(q, dtype=np.complex128).reshape(-1))
        if k.size != nodes or qq.size != nodes or (g is not None and g.size != nodes):
            raise ValueError("kappa, gamma and q need one value per node")
        p = np.zeros(nodes, dtype=np.complex128)
        req = hz.hz_request()
        req.grid = hz.make_grid(dim, n, 1.0 / (n[0] - 1))
        req.kappa = k.ctypes.data
        req.gamma = g.ctypes.data if g is not None else None
        req.gamma0 = float(gamma0)
        req.omega = float(omega)
        req.shift_alpha = float(alpha)
        req.opts = make_opts(dim, levels, **solver_opts)
        req.q = qq.ctypes.data
        req.p = p.ctypes.data
        t = hz.hz_server_submit(self.srv, req)
        self._keep[t] = p           # the server writes here when the request finishes
        return t

    def submit_workload(self, w, k: int = 0, **overrides):
        """Submit source k of a workloads.Workload."""
        opts = dict(patch=w.patch, intergrid=w.intergrid, precision=w.precision, tol=w.tol,
                    restart=w.restart, nu1=w.nu1, nu2=w.nu2, max_iter=w.max_iter,
                    patch_coarse=w.patch_coarse, cycle=w.cycle)
        opts.update(overrides)
        return self.submit(w.dim, w.n, w.kappa, w.omega, w.rhs(k), gamma=w.gamma, alpha=w.alpha,
                           levels=w.levels, **opts)

    def poll(self, ticket) -> dict:
        return _info(hz.hz_server_poll(self.srv, ticket))

    def wait(self, ticket, timeout: float = -1.0):
        """(solution, info dict) once the request has finished or failed."""
        d = _info(hz.hz_server_wait(self.srv, ticket, timeout))
        if self.log is not None and d["state"] in ("done", "failed"):
            self.log.write(request_record(ticket, d))
        return self._keep.pop(ticket), d

    def stats(self) -> dict:
        return hz.hz_server_stats(self.srv)

    def close(self):
        if getattr(self, "srv", None):
            if getattr(self, "log", None) is not None:
                self.log.write(dict(self.stats(), event="server_stats", t=time.time()))
            hz.hz_server_destroy(self.srv)
            self.srv = None
        if getattr(self, "log", None) is not None:
            self.log.close()
            self.log = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def _info(t: hz.hz_ticket_info) -> dict:
    return {"state": hz.REQ_STATE.get(t.state, t.state), "status": hz.STATUS.get(t.status, t.status),
            "iters": t.info.iters, "converged": bool(t.info.converged), "relres_true": t.info.relres_true,
            "t_submit": t.t_submit, "t_admit": t.t_admit, "t_start": t.t_start, "t_done": t.t_done,
            "bytes": t.bytes, "message": t.message.decode(errors="replace"), "group_size": t.group_size}


def request_record(ticket, d: dict) -> dict:
    """The per-request metrics line: end-to-end latency, queueing delay
    (submission to admission), setup span (admission to first restart cycle),
    solve span, iterations, status and device bytes held."""
    rec = {"event": "request", "t": time.time(), "ticket": int(ticket), "state": d["state"], "status": d["status"],
           "iters": d["iters"], "converged": d["converged"], "relres_true": d["relres_true"], "bytes": d["bytes"],
           "group_size": d["group_size"], "latency_s": d["t_done"] - d["t_submit"]}

    def span(a, b):                  # a stage the request never reached has no span
        return d[b] - d[a] if d[b] >= d[a] > 0 or (a == "t_submit" and d[b] >= d[a]) else None
    rec["queue_s"] = span("t_submit", "t_admit")
    rec["setup_s"] = span("t_admit", "t_start")
    rec["solve_s"] = span("t_start", "t_done")
    if d["message"]:
        rec["message"] = d["message"]
    return rec
