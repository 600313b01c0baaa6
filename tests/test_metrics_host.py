"""Per-solve and per-request metrics records (JSON lines), host side: the
fields a solve record carries (iterations, convergence, residuals, restart
history, setup and wall time, V-cycle count, the solver settings), the spans
of a request record, and the sink writing one parseable object per line."""
import io
import json

from paper_2511_16808_gb300 import hz
from paper_2511_16808_gb300.serve import request_record
from paper_2511_16808_gb300.solver import JsonLines, solve_record


def _info(iters, conv, rt, re_):
    i = hz.hz_info()
    i.iters, i.converged, i.relres_true, i.relres_est = iters, conv, rt, re_
    return i


def test_solve_record_fields():
    hist = {"iters": [0, 5, 10, 12], "relres_true": [1.0, 0.2, 3e-4, 8e-7], "relres_est": [1.0, 0.2, 3e-4, 8e-7]}
    rec = solve_record("solve", [_info(12, 1, 8e-7, 7.9e-7)], hist, 0.25, 0.5, 4225, {"levels": 3, "patch": "rb"})
    assert rec["iters"] == [12] and rec["converged"] == [True] and rec["vcycles"] == 12
    assert rec["history"] == hist and rec["setup_s"] == 0.25 and rec["solves_per_s"] == 2.0
    assert rec["levels"] == 3 and rec["patch"] == "rb" and rec["nrhs"] == 1
    batch = solve_record("solve_batch", [_info(7, 1, 1e-7, 1e-7), _info(9, 0, 2e-3, 1e-3)], None, 0.1, 0.0, 10, {})
    assert "history" not in batch and batch["vcycles"] == 16 and batch["solves_per_s"] is None
    assert batch["converged"] == [True, False]


def test_json_lines_sink():
    buf = io.StringIO()
    sink = JsonLines(buf)
    sink.write({"a": 1})
    sink.write({"b": [1.5, None]})
    sink.close()
    lines = buf.getvalue().splitlines()
    assert [json.loads(x) for x in lines] == [{"a": 1}, {"b": [1.5, None]}]


def test_request_record_spans():
    d = {"state": "done", "status": "HZ_OK", "iters": 40, "converged": True, "relres_true": 9e-7, "bytes": 1 << 20,
         "t_submit": 1.0, "t_admit": 1.5, "t_start": 1.75, "t_done": 3.0, "message": "", "group_size": 3}
    r = request_record(7, d)
    assert r["latency_s"] == 2.0 and r["queue_s"] == 0.5 and r["setup_s"] == 0.25 and r["solve_s"] == 1.25
    assert r["group_size"] == 3
    assert "message" not in r and r["ticket"] == 7
    failed = dict(d, state="failed", status="HZ_ERR_INVALID_ARG", t_start=0.0, t_done=1.6, message="kappa")
    r = request_record(8, failed)
    assert r["setup_s"] is None and r["solve_s"] is None and r["queue_s"] == 0.5 and r["message"] == "kappa"
