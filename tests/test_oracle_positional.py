"""Pins of the oracle's positional order (Sec. IV.C): the structure factor
(Eq. 10), the choice of q_0 at its maximum, chi_j (Eq. 11) and the
positional correlation function C_q0(r) (Eq. 12)."""
import numpy as np
import pytest


def square_lattice(n, a):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([i.ravel() * a, j.ravel() * a], axis=1)


def test_structure_factor_of_a_square_lattice(oracle_mod):
    # n x n sites of spacing a = L / n: S = N exactly on the lattice's
    # reciprocal lattice (h, k multiples of n) and 0 at every other point of
    # the box's reciprocal grid (a full sum of n-th roots of unity)
    n, a = 12, 2.3
    L = n * a
    xy = square_lattice(n, a)
    hk = np.array([[n, 0], [0, n], [2 * n, -n], [1, 0], [5, 7], [n, 1], [0, 0]])
    S = oracle_mod.structure_factor(xy, hk, L)
    N = n * n
    assert np.allclose(S[[0, 1, 2, 6]], N, rtol=1e-12)
    assert np.abs(S[[3, 4, 5]]).max() < 1e-18 * N * N + 1e-9


def test_structure_factor_is_translation_invariant(oracle_mod):
    rng = np.random.default_rng(2)
    L = 17.0
    xy = rng.uniform(0, L, (60, 2))
    hk = rng.integers(-6, 7, (20, 2))
    S1 = oracle_mod.structure_factor(xy, hk, L)
    S2 = oracle_mod.structure_factor((xy + [3.3, -7.1]) % L, hk, L)
    assert np.allclose(S1, S2, rtol=1e-10, atol=1e-10)


def test_peak_search_finds_the_reciprocal_vector_of_a_rotated_lattice(oracle_mod):
    # a triangular lattice commensurate with the box: 2 sqrt(3)-ish cell is
    # avoided by using the reciprocal grid directly: pick q0 = 2 pi (h0, k0) / L
    # and positions on the planes q0 . x = 2 pi j; the window search from a
    # guess nearby must return (h0, k0)
    L, h0, k0 = 40.0, 9, 4
    q0 = 2 * np.pi * np.array([h0, k0]) / L
    rng = np.random.default_rng(9)
    # points on lattice planes of q0 (S(q0) = N), randomly placed along them
    t = rng.uniform(0, L, 300)
    j = rng.integers(0, 40, 300)
    e = q0 / np.linalg.norm(q0)
    f = np.array([-e[1], e[0]])
    xy = (np.outer(j * 2 * np.pi / np.linalg.norm(q0), e) + np.outer(t, f)) % L
    window = np.array([[h0 + dh, k0 + dk] for dh in range(-3, 4) for dk in range(-3, 4)])
    hk, S0 = oracle_mod.positional_q0(xy, window, L)
    assert tuple(hk) == (h0, k0) and S0 == pytest.approx(300.0, rel=1e-9)


def test_q0_window_is_centred_on_the_first_shell(oracle_mod):
    # eta and Psi_6 = 1 (bonds along x): centre at angle 30 degrees, |q| = 4 pi / (a sqrt 3)
    eta, L = 0.70, 200.0
    w = oracle_mod.q0_window(1.0 + 0j, eta, L, 0)
    rho = eta / np.pi
    a = np.sqrt(2 / (np.sqrt(3) * rho))
    q = 2 * np.pi * w[0] / L
    assert abs(np.linalg.norm(q) - 4 * np.pi / (a * np.sqrt(3))) < 2 * np.pi / L
    assert abs(np.degrees(np.arctan2(q[1], q[0])) - 30.0) < 1.0
    assert len(oracle_mod.q0_window(1.0 + 0j, eta, L, 2)) == 25


def test_positional_correlation_of_a_lattice_and_a_gas(oracle_mod):
    n, a = 10, 2.2
    L = n * a
    xy = square_lattice(n, a)
    C = oracle_mod.positional_corr(xy, [n, 0], L, [2.2, 4.0, 6.0, 9.0])
    assert np.allclose(C, 1.0, atol=1e-12)  # every pair phase is a multiple of 2 pi
    rng = np.random.default_rng(4)
    gas = rng.uniform(0, 30.0, (900, 2))
    Cg = oracle_mod.positional_corr(gas, [11, 5], 30.0, [3.0, 6.0, 10.0])
    assert np.abs(Cg).max() < 0.05  # ~1/sqrt(pairs in the window)
    # C is real for ordered pairs: (n, m) and (m, n) are conjugate
    assert np.abs(Cg.imag).max() < 1e-12


def test_positional_correlation_windows_against_a_loop(oracle_mod):
    rng = np.random.default_rng(6)
    L = 12.0
    xy = rng.uniform(0, L, (40, 2))
    hk0 = [3, -2]
    q = 2 * np.pi * np.array(hk0) / L
    for r in (1.5, 3.0, 4.5):
        tot, cnt = 0j, 0
        for n in range(40):
            for m in range(40):
                if n == m:
                    continue
                d = xy[n] - xy[m]
                d -= L * np.round(d / L)
                if r - 1.0 <= np.hypot(*d) <= r + 1.0:
                    tot += np.exp(1j * q @ (xy[n] - xy[m]))
                    cnt += 1
        assert abs(oracle_mod.positional_corr(xy, hk0, L, [r])[0] - tot / cnt) < 1e-12
