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
