"""Host check of the error bound behind the FP64 form's float pre-test of a
pair (pair_clear in hd_cell.cuh, bounds set by set_f32_bounds in hd_api.cu).

The device decides a pair in float when the float estimate of d^2 is farther
from 4 than M / 2, the bound on |float estimate - FP64 value|; this test
emulates the same float arithmetic in numpy (the high-word truncation of
approx_f32, float32 round-to-nearest operations without contraction) and
checks the bound on adversarial samples: coordinates at the ends of their
ranges, every cell offset, and pairs near contact."""
import numpy as np
import pytest


def approx_f32(x):
    """High-word truncation of doubles to floats, as approx_f32 does."""
    hi = (np.asarray(x, np.float64).view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    mag = hi & np.uint32(0x7FFFFFFF)
    f = np.where(mag < np.uint32(897 << 20), np.uint32(0), (mag - np.uint32(896 << 20)) << np.uint32(3))
    return (f | (hi & np.uint32(0x80000000))).astype(np.uint32).view(np.float32)


def margin(w, d):
    t, u = 2.0 ** -20, 2.0 ** -24
    R = 2 * w + d
    E = t * (2 * w + d) + u * (3 * w + R)
    return 2 * (4 * R * E + 2 * E * E + 4 * u * (R + E) ** 2 + 16 * 2.0 ** -53 * R * R)


def test_approx_f32_is_a_truncation():
    x = np.array([1.0, -1.0, 3.5, 2.0 ** -126, 2.0 ** -127, 0.0, -0.0, 1.0 + 2.0 ** -20, 1.0 + 2.0 ** -21])
    got = approx_f32(x)
    assert got.tolist() == [1.0, -1.0, 3.5, 2.0 ** -126, 0.0, 0.0, 0.0, 1.0 + 2.0 ** -20, 1.0]
    rng = np.random.default_rng(0)
    y = rng.uniform(-30, 30, 100000)
    rel = np.abs(approx_f32(y).astype(np.float64) - y) / np.abs(y)
    assert rel.max() < 2.0 ** -20
    assert np.all(np.abs(approx_f32(y)) <= np.abs(y))  # toward zero


@pytest.mark.parametrize("w,d", [(2.0008917450904846, 0.1), (2.0122, 0.258), (3.0, 1.4), (7.9, 7.8)])
def test_float_estimate_within_half_margin(w, d):
    rng = np.random.default_rng(1)
    n = 400000
    M = margin(w, d)
    wf = np.float32(w)
    for ox in (-1, 0, 1):
        # coordinates anywhere in their ranges, with a quarter of them pushed to the ends
        qx = rng.uniform(0, w, n)
        qy = rng.uniform(0, w, n)
        px = rng.uniform(-d, w + d, n)
        py = rng.uniform(-d, w + d, n)
        ends = rng.random(n) < 0.25
        qx[ends] = np.nextafter(w, 0)
        px[ends] = -d if ox > 0 else w + d * (1 - 1e-12)
        oy = int(rng.integers(-1, 2))
        # FP64 value as the device computes it (no FMA)
        ax = qx if ox == 0 else qx + (w if ox > 0 else -w)
        ay = qy if oy == 0 else qy + (w if oy > 0 else -w)
        rx, ry = ax - px, ay - py
        d2 = rx * rx + ry * ry
        # float estimate
        fx, fy = approx_f32(qx), approx_f32(qy)
        fax = fx if ox == 0 else (fx + (wf if ox > 0 else -wf)).astype(np.float32)
        fay = fy if oy == 0 else (fy + (wf if oy > 0 else -wf)).astype(np.float32)
        sx = (fax - approx_f32(px)).astype(np.float32)
        sy = (fay - approx_f32(py)).astype(np.float32)
        d2f = (sx * sx).astype(np.float32) + (sy * sy).astype(np.float32)
        err = np.abs(d2f.astype(np.float64) - d2)
        assert err.max() <= M / 2, (err.max(), M)


def test_margin_is_small_at_the_benchmark_geometry():
    # the band that falls back to FP64 stays a tiny slice of the contact shell
    assert margin(2.0008917450904846, 0.1) < 5e-4


def hist_margin(w, H):
    t, u = 2.0 ** -20, 2.0 ** -24
    R = (H + 1) * w
    E = 2 * t * w + u * w * (4 * H + 2)
    return 2 * (4 * R * E + 2 * E * E + 4 * u * (R + E) ** 2 + 16 * 2.0 ** -53 * R * R)


@pytest.mark.parametrize("w,H", [(2.0008917450904846, 2), (2.0122, 2), (1.0 + 2.0 ** -10, 4), (7.9, 1)])
def test_histogram_float_estimate_within_half_margin(w, H):
    """k_hist_tile's FP64 pre-test: both coordinates in [0, w), the
    neighbour H cells away at most, the offset dcx w added in float as
    dcx * wf and in FP64 as a rounded product."""
    rng = np.random.default_rng(2)
    n = 400000
    M = hist_margin(w, H)
    wf = np.float32(w)
    ox = rng.integers(-H, H + 1, n)
    oy = rng.integers(-H, H + 1, n)
    qx, qy = rng.uniform(0, w, n), rng.uniform(0, w, n)
    mx, my = rng.uniform(0, w, n), rng.uniform(0, w, n)
    ends = rng.random(n) < 0.25
    qx[ends] = np.nextafter(w, 0)
    mx[ends] = 0.0
    rx = (qx + ox * w) - mx
    ry = (qy + oy * w) - my
    d2 = rx * rx + ry * ry
    sx = ((approx_f32(qx) + (ox.astype(np.float32) * wf).astype(np.float32)).astype(np.float32) - approx_f32(mx)).astype(np.float32)
    sy = ((approx_f32(qy) + (oy.astype(np.float32) * wf).astype(np.float32)).astype(np.float32) - approx_f32(my)).astype(np.float32)
    d2f = (sx * sx).astype(np.float32) + (sy * sy).astype(np.float32)
    err = np.abs(d2f.astype(np.float64) - d2)
    assert err.max() <= M / 2, (err.max(), M)


def test_library_margins_are_the_checked_bounds(tmp_path):
    """The margins the library computes (hd_bounds.h, compiled here as host
    C++) are the ones whose claim the tests above check."""
    import os
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "margins.cpp"
    src.write_text(
        '#include <cstdio>\n#include "hd_bounds.h"\n'
        "int main() {\n"
        "  const double w[] = {2.0008917450904846, 2.0122, 3.0, 7.9};\n"
        "  const double d[] = {0.1, 0.258, 1.4, 7.8};\n"
        "  const int H[] = {2, 2, 4, 1};\n"
        "  for (int i = 0; i < 4; ++i)\n"
        '    std::printf("%.17g %.17g\\n", hd::pair_f32_margin(w[i], d[i]), hd::cells_f32_margin(w[i], H[i]));\n'
        "}\n")
    exe = tmp_path / "margins"
    subprocess.run([gxx, "-std=c++17", "-O0", "-ffp-contract=off", "-I",
                    os.path.join(root, "paper_1211_1645_gb300", "csrc"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [float(x) for x in out]
    cases = [(2.0008917450904846, 0.1, 2), (2.0122, 0.258, 2), (3.0, 1.4, 4), (7.9, 7.8, 1)]
    for k, (w, d, H) in enumerate(cases):
        assert got[2 * k] == pytest.approx(margin(w, d), rel=1e-14)
        assert got[2 * k + 1] == pytest.approx(hist_margin(w, H), rel=1e-14)
