"""The request server's grouping policy on the CPU (server_policy.h compiled
for the host with g++): the host-staging cap of a group, power-of-two group
sizes from the queued candidates, the HBM budget (the leader's bytes replaced
by the group's), and a refused size keeping the request alone."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_grouping_policy(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path / "group_policy_check")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I",
                        os.path.join(ROOT, "paper_2511_16808_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "group_policy_check.cpp"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([out], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
