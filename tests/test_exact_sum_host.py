"""Host check (no GPU) of the exact sum behind the device's global Psi_6
(hd_exact.cuh): a host-only build of the same header sums seeded and
adversarial doubles, and the rounded result is compared with exact
rational arithmetic (fractions.Fraction, rounded once by float()), in file
order and in chunks merged in reverse order."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1211_1645_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("exact") / "exact_sum_host")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I" + CSRC, "-o", out,
                           os.path.join(HERE, "host", "exact_sum_host.cu")])
    return out


def run(harness, tmp_path, values, chunk=7):
    f = tmp_path / "v.bin"
    f.write_bytes(np.asarray(values, dtype="<f8").tobytes())
    a, b = subprocess.check_output([harness, str(f), str(chunk)]).split()
    return [struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0] for h in (a, b)]


def exact(values):
    return float(sum((Fraction(float(v)) for v in values), Fraction(0)))


def same(x, y):
    return struct.pack("<d", x) == struct.pack("<d", y) or (x == y == 0.0)


CASES = {
    "uniform": np.random.default_rng(0).uniform(-1, 1, 20000),
    "psi_like_small_mean": np.random.default_rng(1).uniform(-1, 1, 20000) * 1e-3 + 1e-7,
    "wide_exponents": (np.random.default_rng(2).choice([-1.0, 1.0], 5000)
                       * 2.0 ** np.random.default_rng(3).integers(-75, 61, 5000)),
    "cancellation": [1e10, 1.0, -1e10, 2.0 ** -70, -3.0],
    "tie_to_even_down": [1.0, 2.0 ** -53],
    "tie_to_even_up": [1.0 + 2.0 ** -52, 2.0 ** -53],
    "just_above_tie": [1.0, 2.0 ** -53, 2.0 ** -75],
    "negative_tie": [-1.0, -(2.0 ** -53), -(2.0 ** -53), 2.0 ** -53],
    "sum_zero": [0.5, -0.25, -0.25],
    "small_only": [2.0 ** -75, 3 * 2.0 ** -75, -(2.0 ** -74)],
    "large_terms": [2.0 ** 61, 2.0 ** 61, -(2.0 ** 60), 1.0],
    "carry_chains": [2.0 ** -64, -(2.0 ** -64), 2.0 ** -1, 2.0 ** -75, -(2.0 ** -75), -(2.0 ** -1)],
}


@pytest.mark.parametrize("case", list(CASES))
def test_exact_sum_is_exactly_rounded(harness, tmp_path, case):
    v = CASES[case]
    a, b = run(harness, tmp_path, v)
    want = exact(v)
    assert same(a, want), (a, want)
    assert same(b, want), (b, want)


def test_tiny_terms_truncated_and_nonfinite_marks_invalid(harness, tmp_path):
    # below 2^-128 a term is truncated toward zero (documented resolution)
    a, _ = run(harness, tmp_path, [2.0 ** -1074, 2.0 ** -130, -(2.0 ** -129)])
    assert a == 0.0
    a, b = run(harness, tmp_path, [1.0, float("nan")])
    assert np.isnan(a) and np.isnan(b)
    a, _ = run(harness, tmp_path, [2.0 ** 62])
    assert np.isnan(a)


def test_order_independent_bits(harness, tmp_path):
    rng = np.random.default_rng(4)
    v = rng.standard_normal(5000) * 2.0 ** rng.integers(-60, 20, 5000)
    a, b = run(harness, tmp_path, v, chunk=1)
    c, d = run(harness, tmp_path, v[::-1], chunk=333)
    assert same(a, b) and same(a, c) and same(a, d)
    assert same(a, exact(v))
