"""The CUDA path's integer-pipe float <-> double conversions, bit for bit, and
its error-free FP32 neighbour sums against exactly rounded sums.

The FP64 Krylov passes widen FP32 vectors and the mixed V-cycle narrows FP64
ones with integer operations only (the hardware conversion runs on the slow
FP64 pipe of this GPU).  The same source is compiled for the host here and
checked against numpy's IEEE conversions (exact widening; round to nearest
even with subnormal results and overflow to infinity) on every class of
input: zeros, all float subnormal patterns, normals, the overflow and
underflow boundaries, exact ties, infinities and NaNs.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def conv_bin(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("conv") / "conv_check"
    src = os.path.join(ROOT, "tests", "conv_check.cu")
    inc = os.path.join(ROOT, "paper_2511_16808_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-I", inc, "-I", os.path.join(ROOT, "include"),
                        src, "-o", str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(out)


def _run(binary, f32, f64, tmp):
    a, b, c, d = (os.path.join(tmp, n) for n in ("a.bin", "b.bin", "c.bin", "d.bin"))
    f32.tofile(a)
    f64.tofile(c)
    subprocess.run([binary, a, b, c, d], check=True)
    return np.fromfile(b, dtype=np.float64), np.fromfile(d, dtype=np.float32)


def _float_patterns():
    rng = np.random.default_rng(0)
    sub = np.arange(0, 1 << 23, 7, dtype=np.uint32)                    # subnormals (and 0)
    sub = np.concatenate([sub, np.arange(1, 64, dtype=np.uint32), np.uint32([(1 << 23) - 1])])
    rnd = rng.integers(0, 1 << 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    special = np.uint32([0x7f800000, 0x7f800001, 0x7fc00000, 0x7fffffff, 0x00800000, 0x7f7fffff, 0x3f800000])
    u = np.concatenate([sub, rnd, special])
    u = np.concatenate([u, u | np.uint32(0x80000000)])
    return u.view(np.float32)


def _double_patterns():
    rng = np.random.default_rng(1)
    n = 1 << 19
    mant = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    parts = []
    # exponents spanning float underflow to overflow, plus the rest of the range
    for lo, hi in ((1023 - 160, 1023 - 120), (1023 - 126, 1023 + 128), (0, 2047)):
        e = rng.integers(lo, hi, size=n, dtype=np.uint64)
        parts.append((e << np.uint64(52)) | mant)
    # exact ties and near-ties at the 29-bit rounding position and in the subnormal range
    e = rng.integers(1023 - 149, 1023 + 127, size=n, dtype=np.uint64)
    keep = mant & ~np.uint64((1 << 29) - 1)
    for t in (1 << 28, (1 << 28) - 1, (1 << 28) + 1):
        parts.append((e << np.uint64(52)) | keep | np.uint64(t))
    es = rng.integers(1023 - 152, 1023 - 126, size=n, dtype=np.uint64)
    for t in range(30, 54):
        parts.append((es << np.uint64(52)) | (mant & ~np.uint64((1 << t) - 1)) | np.uint64(1 << (t - 1)))
    special = np.array([0, 1, (1 << 52) - 1, 0x7ff0000000000000, 0x7ff8000000000000, 0x7ff0000000000001,
                        0x47efffffe0000000, 0x47efffffefffffff, 0x47effffff0000000, 0x36a0000000000000,
                        0x3690000000000000, 0x3690000000000001, 0x380fffffffffffff, 0x3810000000000000],
                       dtype=np.uint64)
    u = np.concatenate(parts + [special])
    u = np.concatenate([u, u | np.uint64(1 << 63)])
    return u.view(np.float64)


def test_widening_is_exact(conv_bin, tmp_path):
    f = _float_patterns()
    wide, _ = _run(conv_bin, f, np.zeros(1), str(tmp_path))
    with np.errstate(invalid="ignore"):
        ref = f.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(wide[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    assert np.all(np.isnan(wide[nan]))
    # NaN payloads carried over (quiet bit set by the source pattern or kept)
    fb = f[nan].view(np.uint32).astype(np.uint64)
    wb = wide[nan].view(np.uint64)
    assert np.array_equal((wb >> np.uint64(29)) & np.uint64((1 << 23) - 1), fb & np.uint64((1 << 23) - 1))


def test_narrowing_rounds_to_nearest_even(conv_bin, tmp_path):
    d = _double_patterns()
    _, narrow = _run(conv_bin, np.zeros(1, dtype=np.float32), d, str(tmp_path))
    with np.errstate(over="ignore", invalid="ignore"):
        ref = d.astype(np.float32)
    nan = np.isnan(ref)
    assert np.array_equal(narrow[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    assert np.all(np.isnan(narrow[nan]))
    # signed zeros / infinities / subnormal results are all present in the sample
    assert np.any(ref[~nan] == 0) and np.any(np.isinf(ref)) and np.any((ref != 0) & (np.abs(ref) < 1.1754944e-38))


def test_neighbour_sums_within_bound(conv_bin, tmp_path):
    """fsum_wide (FP32 two-sums + one FP64 add) against math.fsum of the same
    values: |error| <= (n-1)^2 2^-48 max partial sum, on random values of
    mixed magnitudes and on sets built to cancel."""
    import math
    rng = np.random.default_rng(7)
    m = 20000
    g = rng.standard_normal((m, 6)) * 10.0 ** rng.integers(-6, 7, size=(m, 6))
    g[: m // 4, 1] = -g[: m // 4, 0] * (1 + 1e-7 * rng.standard_normal(m // 4))   # near cancellation
    g[m // 4: m // 2, 5] = -g[m // 4: m // 2, :5].sum(axis=1)
    f = g.astype(np.float32)
    inp = os.path.join(str(tmp_path), "s.bin")
    out = os.path.join(str(tmp_path), "r.bin")
    f.tofile(inp)
    subprocess.run([conv_bin, "--sum", inp, out], check=True)
    r = np.fromfile(out, dtype=np.float64).reshape(m, 2)
    for k, n in ((0, 4), (1, 6)):
        vals = f[:, :n].astype(np.float64)
        exact = np.array([math.fsum(row) for row in vals])
        partial = np.max(np.abs(np.cumsum(vals, axis=1)), axis=1)
        bound = (n - 1) ** 2 * 2.0 ** -48 * partial
        assert np.all(np.abs(r[:, k] - exact) <= bound), np.max(np.abs(r[:, k] - exact) / np.maximum(bound, 1e-300))


@pytest.mark.parametrize("k", [0, 14, 20, 120])
def test_power_of_two_widening_is_exact(conv_bin, tmp_path, k):
    """f2d_exact_pow2(f, k) is the exact f * 2^k (the operator's 1/h^2 = 2^k
    folded into the widening), for every class of float input."""
    f = _float_patterns()
    inp = os.path.join(str(tmp_path), "f.bin")
    out = os.path.join(str(tmp_path), "w.bin")
    f.tofile(inp)
    subprocess.run([conv_bin, "--pow2", str(k), inp, out], check=True)
    w = np.fromfile(out, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        ref = np.ldexp(f.astype(np.float64), k)
    nan = np.isnan(ref)
    assert np.array_equal(w[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    assert np.all(np.isnan(w[nan]))


@pytest.mark.parametrize("k", [10, 20])
def test_power_of_two_neighbour_sums_match_scaled(conv_bin, tmp_path, k):
    """fsum_wide_pow2(v, k) == 2^k fsum_wide(v) bit for bit: the operator's
    interior rows give the same FP64 result with and without the folding."""
    rng = np.random.default_rng(11)
    m = 20000
    g = rng.standard_normal((m, 6)) * 10.0 ** rng.integers(-30, 30, size=(m, 6))
    g[: m // 4, 1] = -g[: m // 4, 0] * (1 + 1e-7 * rng.standard_normal(m // 4))
    f = g.astype(np.float32)
    f[m // 2: m // 2 + 100] = np.float32(1e-44)                   # float subnormals
    inp = os.path.join(str(tmp_path), "s.bin")
    a = os.path.join(str(tmp_path), "a.bin")
    b = os.path.join(str(tmp_path), "b.bin")
    f.tofile(inp)
    subprocess.run([conv_bin, "--sum", inp, a], check=True)
    subprocess.run([conv_bin, "--sum-pow2", str(k), inp, b], check=True)
    plain = np.fromfile(a, dtype=np.float64)
    folded = np.fromfile(b, dtype=np.float64)
    assert np.array_equal(folded.view(np.uint64), np.ldexp(plain, k).view(np.uint64))
