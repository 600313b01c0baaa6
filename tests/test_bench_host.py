"""Host-side pieces of the measurement tools: the constant stencil that the
LFA bench mode feeds the library equals the oracle's 5-/7-point stencil at the
same shift, and the command-line modules import without a device."""
import importlib

import numpy as np
import pytest

import bench
from oracle import operator


@pytest.mark.parametrize("dim,n", [(2, 513), (3, 129)])
def test_lfa_bench_stencil_is_the_shifted_operator(dim, n):
    st = bench._lfa_stencil(dim, n, alpha=0.2)
    h = 1.0 / (n - 1)
    omega = 2 * np.pi / (10.0 * h)
    ref = operator.five_point_stencil(h, omega ** 2 * (1 - 0.01j) - 0.2j * omega ** 2, dim)
    assert set(st) == set(ref)
    for k in ref:
        assert abs(st[k] - ref[k]) <= 1e-12 * abs(ref[k])


@pytest.mark.parametrize("mod", ["paper_2511_16808_gb300.tables",
                                 "paper_2511_16808_gb300.tuning", "paper_2511_16808_gb300.serve"])
def test_modules_import_without_device(mod):
    m = importlib.import_module(mod)
    assert m.__doc__


def test_reference_arm_line():
    """`bench.py --impl reference` (the oracle on one host core) prints one JSON
    line with the contract's keys; e2e repeats the value with no host-device
    bytes, cpu_baseline describes the run."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--config", "config1",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["higher_is_better"] is True
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["kind"] == "oracle"
