"""Pins of the oracle's psi_6 autocorrelation (Sec. III, Eq. 9) and the
correlation time from its exponential part (Table II's tau)."""
import numpy as np
import pytest


def test_constant_series_is_fully_correlated(oracle_mod):
    # C(dt) = 1 at every lag: catches averaging the numerator over T instead
    # of the T - dt available pairs, and a denominator of |Psi| instead of |Psi|^2
    z = np.full(50, 0.3 - 0.4j)
    C = oracle_mod.psi6_acf(z, 20)
    assert np.allclose(C, 1.0, rtol=0, atol=1e-15)


def test_uniform_rotation_gives_a_pure_phase(oracle_mod):
    # Psi(t) = A exp(i w t): Psi(t) Psi*(t + dt) = |A|^2 exp(-i w dt) for every t,
    # so C(dt) = exp(-i w dt) exactly (fixes which factor is conjugated)
    w, A = 0.37, 0.2 + 0.1j
    t = np.arange(400)
    z = A * np.exp(1j * w * t)
    C = oracle_mod.psi6_acf(z, 60)
    assert np.abs(C - np.exp(-1j * w * np.arange(61))).max() < 1e-12


def test_ar1_process_decays_as_rho_to_the_lag(oracle_mod):
    # stationary complex AR(1): z(t+1) = rho z(t) + sqrt(1 - rho^2) xi(t),
    # E|xi|^2 = 1, has C(dt) = rho^dt and tau = -1 / ln rho
    rho, T = 0.9, 200_000
    rng = np.random.default_rng(11)
    xi = (rng.standard_normal(T) + 1j * rng.standard_normal(T)) / np.sqrt(2.0)
    z = np.empty(T, complex)
    z[0] = xi[0]
    a = np.sqrt(1.0 - rho * rho)
    for t in range(1, T):
        z[t] = rho * z[t - 1] + a * xi[t]
    C = oracle_mod.psi6_acf(z, 20)
    # standard error of C(dt) ~ sqrt((1 + rho^2) / ((1 - rho^2) T)) ~ 0.007
    assert np.abs(C.real - rho ** np.arange(21)).max() < 0.04
    assert np.abs(C.imag).max() < 0.04
    tau = oracle_mod.acf_tau(C, 1, 10)
    assert abs(tau / (-1.0 / np.log(rho)) - 1.0) < 0.05


def test_tau_of_an_exact_exponential(oracle_mod):
    tau = 123.25
    d = np.arange(200)
    C = np.exp(-d / tau) * (1 + 0j)
    assert abs(oracle_mod.acf_tau(C, 5, 150) - tau) < 1e-9 * tau
    # lags where C <= 0 are not in the fit; too few lags give NaN
    C2 = C.copy()
    C2[100:] = -0.01
    assert abs(oracle_mod.acf_tau(C2, 5, 150) - tau) < 1e-9 * tau
    assert np.isnan(oracle_mod.acf_tau(C2, 120, 150))
    # a growing "decay" is not a correlation time
    assert np.isnan(oracle_mod.acf_tau(np.exp(d / tau) + 0j, 1, 50))


def test_lag_range_is_checked(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.psi6_acf(np.ones(5), 5)
