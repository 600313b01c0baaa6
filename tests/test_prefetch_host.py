"""The clipping of the kernels' L2 prefetches, on the CPU: the same
plane_row_run the device code uses, compiled for the host, on 20000 seeded
random grids and block regions (2D and one z plane of 3D grids): every
prefetched element run lies inside the stencil planes and the runs cover the
block region clipped to the grid exactly once."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_prefetch_runs_stay_inside_and_cover(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path / "prefetch_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I", os.path.join(ROOT, "paper_2511_16808_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "prefetch_check.cu"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([out], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.startswith("ok"), run.stdout + run.stderr
