"""Pins of the oracle's pressure estimator (Eqs. 2 and 4, quartic contact
extrapolation of Sec. II.C.1) against closed forms: exact polynomial
recovery, ideal-gas g(r), the exact two-disk pressure from d ln Z / dV and
the hard-disk virial series."""
import os

import numpy as np
import pytest

from helpers import batch_se

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hard_disk_virial.txt")


def _virial():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v, kind = line.split()
            out[int(k)] = (float(v), kind)
    return out


def test_virial_golden_closed_forms():
    v = _virial()
    assert v[3][0] == pytest.approx(4 / 3 - np.sqrt(3) / np.pi, abs=1e-8)
    assert v[4][0] == pytest.approx(2 - 4.5 * np.sqrt(3) / np.pi + 10 / np.pi ** 2, abs=1e-8)


def test_quartic_fit_exact(oracle_mod):
    r = 2.0 + (np.arange(100) + 0.5) * 1e-3
    x = r - 2.0
    coef = [6.675, -41.3, 310.0, -2500.0, 9000.0]
    g = sum(c * x ** p for p, c in enumerate(coef))
    assert oracle_mod.contact_fit(r, g) == pytest.approx(coef[0], rel=1e-12)


def test_ideal_gas_g_is_flat(oracle_mod):
    """Uniform independent points: the expected number of pairs per shell is
    (N(N-1)/2) 2 pi r dr / V, so with p = N^2/2 Eq. 2 gives g = (N-1)/N."""
    N = 2000
    L = 100.0
    o = oracle_mod.OracleChain(N, N * np.pi / L ** 2, 0.1, 1, form="fp64")
    assert o.geometry()["L"] == pytest.approx(L, rel=1e-14)
    rng = np.random.default_rng(7)
    K, dr = 50, 0.01
    g0s, gall = [], []
    for _ in range(80):
        o.set_positions(rng.uniform(0, L, size=(N, 2)))
        h = o.histogram(K, dr)
        assert np.array_equal(h, o.histogram(K, dr, brute=True))
        r, g = oracle_mod.g_of_r(h, N, L, dr)
        gall.append(g)
        g0s.append(oracle_mod.contact_fit(r, g))
    want = (N - 1) / N
    m, se = np.mean(g0s), np.std(g0s, ddof=1) / np.sqrt(len(g0s))
    assert abs(m - want) < 4 * se
    gbar = np.mean(gall, axis=0)
    assert abs(gbar.mean() - want) < 0.01


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_two_disk_pressure_exact(oracle_mod, form):
    """Two disks, V = 100: Z ~ V (V - 4 pi sigma^2), so beta P = 1/V +
    1/(V - 4 pi); Eq. 4 with p = N^2/2 must reproduce it.  (With p = N(N-1)/2
    the estimate would be 1 + 2 eta g larger by a factor 2 in g.)"""
    eta = 2 * np.pi / 100.0
    o = oracle_mod.OracleChain(2, eta, 1.0, 777, form=form)
    g = o.geometry()
    L, V = g["L"], g["L"] ** 2
    K, dr = 45, 0.01
    dr_real = o.realised_dr(dr)
    o.sweep(200)
    nb, per = 20, 4000
    est = []
    tot = np.zeros(K, np.float64)
    for b in range(nb):
        acc = np.zeros(K, np.float64)
        for _ in range(per):
            o.sweep(2)
            acc += o.histogram(K, dr)
        tot += acc
        est.append(oracle_mod.contact_pressure(acc / per, 2, L, dr_real)["betaP_over_rho"])
    exact = (V / 2.0) * (1.0 / V + 1.0 / (V - 4 * np.pi))
    got = oracle_mod.contact_pressure(tot / (nb * per), 2, L, dr_real)["betaP_over_rho"]
    se = np.std(est, ddof=1) / np.sqrt(nb)
    assert abs(got - exact) < 4 * se + 1e-4, (got, exact, se)
    # the wrong pair normalisation is far outside the error bar
    wrong = 1.0 + 2 * (got - 1.0)
    assert abs(wrong - exact) > 5 * se


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_virial_series_low_density(oracle_mod, form):
    """beta P / rho at eta = 0.1 against the virial series through B4
    (B5, B6 bound the truncation), N = 1024 disks."""
    v = _virial()
    eta = 0.1
    y = 2 * eta
    p_b4 = 1 + y + v[3][0] * y ** 2 + v[4][0] * y ** 3
    tail = v[5][0] * y ** 4 + v[6][0] * y ** 5
    o = oracle_mod.OracleChain(1024, eta, 0.7, 2024, form=form)
    g = o.geometry()
    K, dr = 100, 1e-3
    dr_real = o.realised_dr(dr)
    o.sweep(500)
    samples = []
    for _ in range(6000):
        o.sweep(3)
        samples.append(o.histogram(K, dr))
    samples = np.array(samples, dtype=np.float64)
    nb = 20
    est = [oracle_mod.contact_pressure(b.mean(0), 1024, g["L"], dr_real)["betaP_over_rho"]
           for b in np.array_split(samples, nb)]
    got = oracle_mod.contact_pressure(samples.mean(0), 1024, g["L"], dr_real)["betaP_over_rho"]
    se = np.std(est, ddof=1) / np.sqrt(nb)
    assert se < 0.005
    assert abs(got - p_b4) < 4 * se + 1.5 * tail, (got, p_b4, se)
    # the second virial coefficient alone is excluded
    assert abs(got - (1 + y)) > 4 * se
