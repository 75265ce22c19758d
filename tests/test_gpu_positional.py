"""GPU parity of the positional-order analysis (Sec. IV.C, Eqs. 10-12)
against the oracle on the same chain states."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import paper_1211_1645_gb300 as hd
    hd.load()
    return hd


def pair(hd, oracle_mod, form, N=1000, eta=0.70, seed=12, sweeps=20):
    g = hd.HardDisks(N, eta, 0.12, seed, precision=form)
    o = oracle_mod.OracleChain(N, eta, 0.12, seed, form=form)
    g.sweep(sweeps)
    o.sweep(sweeps)
    geo = o.geometry()
    L = geo["LF"] / oracle_mod.FX_SCALE if form == "fixed" else geo["L"]
    assert np.array_equal(g.positions(), o.positions())
    return g, o, L


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_structure_factor(hd, oracle_mod, form):
    g, o, L = pair(hd, oracle_mod, form)
    rng = np.random.default_rng(3)
    hk = rng.integers(-40, 41, (37, 2))
    hk[0] = [0, 0]
    S = g.structure_factor(hk)[0]
    want = oracle_mod.structure_factor(o.positions(), hk, L)
    assert S[0] == pytest.approx(1000.0, rel=1e-12)  # S(0) = N
    assert np.abs(S - want).max() <= 1e-9 * max(1.0, want.max())
    g.close()


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_q0_field_and_correlation(hd, oracle_mod, form):
    g, o, L = pair(hd, oracle_mod, form, N=1600, eta=0.72, sweeps=30)
    hk0, S0 = g.positional_q0(3)
    _, psi = o.psi6()
    glob = o.psi6()[1]
    eta = o.N * np.pi / (L * L)
    window = oracle_mod.q0_window(glob, eta, L, 3)
    want_hk, want_S = oracle_mod.positional_q0(o.positions(), window, L)
    assert tuple(hk0[0]) == tuple(want_hk)
    assert S0[0] == pytest.approx(want_S, rel=1e-9)

    chi = oracle_mod.positional_chi(o.positions(), hk0[0], L)
    f = g.positional_field(hk0[0], 6)[0]
    want_f = oracle_mod.psi6_field(o.positions(), chi, L, 6, LF=o.geometry()["LF"] if form == "fixed" else None)
    assert np.array_equal(np.isnan(f.real), np.isnan(want_f.real))
    ok = ~np.isnan(want_f.real)
    assert np.abs(f[ok] - want_f[ok]).max() <= 1e-9

    nr, dr = 14, 0.5
    C = g.positional_corr(hk0[0], nr, dr)[0]
    want_C = oracle_mod.positional_corr(o.positions(), hk0[0], L, (np.arange(nr) + 1) * dr)
    empty = np.isnan(want_C.real)
    assert np.array_equal(np.isnan(C.real), empty)
    assert empty[0] and empty[1]  # no pair closer than 2 sigma: windows up to r = 1 sigma are empty
    assert np.abs(C[~empty] - want_C[~empty]).max() <= 1e-9
    assert np.abs(C[~empty].imag).max() <= 1e-9  # ordered pairs: a real function
    g.close()


def test_positional_errors(hd):
    from paper_1211_1645_gb300.hd import HD_ERR_ARG, HD_ERR_REACH, HDError
    g = hd.HardDisks(256, 0.70, 0.1, 1, precision="fixed")
    with pytest.raises(HDError) as e:
        g.positional_corr([4, 0], 200, 0.5)  # r = 100 sigma: the cell reach wraps a 34 sigma box
    assert e.value.status == HD_ERR_REACH
    with pytest.raises(HDError) as e:
        g.positional_corr([4, 0], 0, 0.5)
    assert e.value.status == HD_ERR_ARG
    with pytest.raises(HDError) as e:
        g.structure_factor(np.zeros((0, 2), int))
    assert e.value.status == HD_ERR_ARG
    g.close()
