"""Per-solve metrics on the GPU: the restart history recorded by the library,
the setup time, and the JSON lines written by the solver and the server.

- The history starts at (0 iterations, relative residual 1) and ends at the
  solve's own iteration count and true residual; one entry per restart cycle
  in between (ceil(iters / m) cycles), iterations increasing.
- A solver with log= writes one parseable line per solve with that history.
- A batched solve clears the history.
- A server with log= writes one line per finished request and a closing line
  with its counters; the spans add up to the latency.
"""
import io
import json
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pairs import medium  # noqa: E402


def _solver(log=None, nrhs_max=1):
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    h, omega, kappa, gamma = medium(2, 65, 0, 8)
    return HelmholtzSolver(2, [65, 65], kappa, omega, gamma, 0.25, 3, patch="rb", intergrid="leveldep",
                           precision="mixed", tol=1e-7, log=log, nrhs_max=nrhs_max), h


def _source(h, node=(32, 32)):
    import workloads
    return workloads.point_source((65, 65), node, h).ravel()


def test_history_and_solve_log():
    buf = io.StringIO()
    s, h = _solver(log=buf)
    p, info = s.solve(torch.tensor(_source(h), device="cuda"))
    hist = s.history()
    assert s.setup_seconds() > 0
    its, rt = hist["iters"], hist["relres_true"]
    assert its[0] == 0 and abs(rt[0] - 1.0) < 1e-12
    assert its[-1] == info.iters and rt[-1] == info.relres_true and rt[-1] < 1e-7
    assert len(its) == 1 + math.ceil(info.iters / 5) and its == sorted(its)
    rec = json.loads(buf.getvalue().splitlines()[-1])
    assert rec["event"] == "solve" and rec["iters"] == [info.iters] and rec["history"] == hist
    assert rec["setup_s"] > 0 and rec["wall_s"] > 0 and rec["patch"] == "rb" and rec["levels"] == 3
    s.close()


def test_batched_solve_clears_history():
    s, h = _solver(nrhs_max=2)
    s.solve(torch.tensor(_source(h), device="cuda"))
    assert len(s.history()["iters"]) >= 2
    Q = torch.tensor(np.stack([_source(h), _source(h, (20, 40))], axis=1), device="cuda")
    s.solve_batch(Q)
    assert s.history()["iters"] == []
    s.close()


def test_server_log():
    from paper_2511_16808_gb300.serve import Server
    buf = io.StringIO()
    h, omega, kappa, gamma = medium(2, 65, 0, 8)
    with Server(max_active=2, log=buf) as srv:
        ts = [srv.submit(2, 65, kappa, omega, _source(h, node), gamma=gamma, alpha=0.25, levels=3, patch="rb",
                         intergrid="leveldep", tol=1e-7) for node in ((32, 32), (10, 50))]
        res = [srv.wait(t, timeout=300) for t in ts]
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    reqs = [x for x in lines if x["event"] == "request"]
    assert len(reqs) == 2 and lines[-1]["event"] == "server_stats" and lines[-1]["done"] == 2
    for r, (_, d) in zip(reqs, res):
        assert r["iters"] == d["iters"] and r["status"] == "HZ_OK"
        assert r["queue_s"] >= 0 and r["setup_s"] >= 0 and r["solve_s"] >= 0
        assert abs(r["queue_s"] + r["setup_s"] + r["solve_s"] - r["latency_s"]) < 1e-9


def test_measured_arithmetic_peaks_are_plausible():
    """The chain kernel's FP64 and FP32 rates: positive, FP64 at most the
    nominal figure of 152 SMs x 2 DFMA lanes x 2 flops x 2.07 GHz (5% margin
    for clock reporting), and FP32 far above FP64 on this part."""
    from paper_2511_16808_gb300 import hz
    t64, ms64 = hz.hz_measure_peak("fp64")
    t32, ms32 = hz.hz_measure_peak("fp32")
    assert ms64 > 0 and ms32 > 0
    props = torch.cuda.get_device_properties(0)
    nominal64 = props.multi_processor_count * 2 * 2 * 2.07e9 / 1e12
    assert 0.2 * nominal64 < t64 < 1.05 * nominal64, (t64, nominal64)
    assert t32 > 8 * t64, (t32, t64)
    with pytest.raises(hz.HzError):
        hz.hz_measure_peak(7)
