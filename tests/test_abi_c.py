"""The C ABI from plain C: tests/abi_c_check.c is compiled with gcc -std=c99
-Wall -Wextra -Werror against include/hz.h, linked to the built libhz.so and
run (device-free calls only: version, defaults, size estimates, option and
argument checks)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_consumer(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_2511_16808_gb300 import build
    lib = build.LIB
    if not os.path.exists(lib):
        build.build()
    exe = tmp_path / "abi_c_check"
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "abi_c_check.c"), "-o", str(exe), "-L", libdir, "-lhz",
           f"-Wl,-rpath,{libdir}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
