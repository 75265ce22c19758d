"""Pins of the oracle's coarse-grained psi_6 field: means of psi_j over
bins x bins square sampling areas of side L / bins (Figs. 5-6)."""
import numpy as np


def test_uniform_local_order_gives_a_uniform_field(oracle_mod):
    rng = np.random.default_rng(3)
    L, n = 20.0, 300
    xy = rng.uniform(0, L, (n, 2))
    c = 0.25 - 0.625j  # dyadic: every partial sum and the division are exact
    f = oracle_mod.psi6_field(xy, np.full(n, c), L, 7)
    full = ~np.isnan(f.real)
    assert full.sum() > 40
    assert np.all(f[full] == c)


def test_one_area_is_the_global_mean(oracle_mod):
    rng = np.random.default_rng(4)
    xy = rng.uniform(0, 10.0, (101, 2))
    psi = rng.standard_normal(101) + 1j * rng.standard_normal(101)
    f = oracle_mod.psi6_field(xy, psi, 10.0, 1)
    assert abs(f[0, 0] - psi.mean()) < 1e-14


def test_areas_are_half_open(oracle_mod):
    # a centre on an area edge belongs to the area above it; [iy, ix] indexing
    L, bins = 8.0, 4
    xy = np.array([[2.0, 0.5], [np.nextafter(2.0, 0.0), 0.5], [0.0, 6.0], [7.999, 7.999]])
    psi = np.array([1.0, 2.0, 3.0, 4.0]) + 0j
    f = oracle_mod.psi6_field(xy, psi, L, bins)
    assert f[0, 1] == 1.0 and f[0, 0] == 2.0 and f[3, 0] == 3.0 and f[3, 3] == 4.0
    assert np.isnan(f[1, 1].real)


def test_fixed_point_areas_use_the_exact_integer_coordinate(oracle_mod):
    # box side LF = 3 * 2^24 + 1 units: X bins // LF differs from a float
    # formula only by exact rounding; coordinates on the grid 2^-24
    LF = 3 * (1 << 24) + 1
    L = LF / oracle_mod.FX_SCALE
    bins = 3
    X = np.array([[LF // 3, 5], [LF // 3 + 1, 5], [LF - 1, LF - 1]], dtype=np.int64)
    # X bins // LF: (LF // 3) * 3 < LF -> area 0; (LF // 3 + 1) * 3 >= LF -> area 1
    xy = X / oracle_mod.FX_SCALE
    psi = np.array([1.0, 2.0, 3.0]) + 0j
    f = oracle_mod.psi6_field(xy, psi, L, bins, LF=LF)
    assert f[0, 0] == 1.0 and f[0, 1] == 2.0 and f[2, 2] == 3.0


def test_against_a_loop_over_areas(oracle_mod):
    rng = np.random.default_rng(5)
    L, bins, n = 13.0, 6, 500
    xy = rng.uniform(0, L, (n, 2))
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    f = oracle_mod.psi6_field(xy, psi, L, bins)
    side = L / bins
    for iy in range(bins):
        for ix in range(bins):
            sel = ((xy[:, 0] >= ix * side) & (xy[:, 0] < (ix + 1) * side) &
                   (xy[:, 1] >= iy * side) & (xy[:, 1] < (iy + 1) * side))
            if sel.any():
                assert abs(f[iy, ix] - psi[sel].mean()) < 1e-13
            else:
                assert np.isnan(f[iy, ix].real)
