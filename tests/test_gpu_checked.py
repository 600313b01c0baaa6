"""The checked-index debug build (libhz_checked.so, hz_check_status).

Built with -DHZ_CHECKED, every instrumented global access of the solve's
kernels (stencil neighbours and coefficient planes of every level, tile
loads and stores of the fused passes, transfers, the coarsest product, the
FP64 Krylov passes) tests its index against the array's extent and counts an
access outside it instead of making it.  A child process loads that library
(HZ_LIB) and solves 2D and 3D cases with every patch type, both precisions,
the compact stencil, a W-cycle and a 16-RHS batch (tensor-core coarsest
product); each must agree with the oracle at the same tolerance, and the
library must report zero out-of-extent accesses.  The normal library reports
the check as disabled.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_normal_library_reports_check_disabled():
    from paper_2511_16808_gb300 import hz
    st = hz.hz_check_status()
    assert st["enabled"] is False and st["failures"] == 0


def test_checked_build_runs_clean():
    from paper_2511_16808_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, HZ_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env, capture_output=True,
                       text=True, timeout=1500)
    print(r.stdout[-6000:])
    print(r.stderr[-3000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert '"enabled": true' in r.stdout and '"failures": 0' in r.stdout
