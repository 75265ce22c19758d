"""GPU parity of the analysis calls against the oracle: the Psi_6
autocorrelation (Eq. 9) and correlation time of the recorded series, and the
coarse-grained psi_6 field of the current state."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PSI_TOL = {"fp64": 1e-12, "fixed": 2.5e-7}


@pytest.fixture(scope="module")
def hd():
    import paper_1211_1645_gb300 as hd
    hd.load()
    return hd


def series_psi(g):
    s = g.series()  # [T, R, 4]
    return s[:, :, 2] + 1j * s[:, :, 3]


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_acf_and_tau_match_the_oracle_on_the_recorded_series(hd, oracle_mod, form):
    g = hd.HardDisks([400, 1000, 576], [0.70, 0.72, 0.65], [0.15] * 3, [3, 4, 5], precision=form)
    g.series_reserve(200)
    g.run(90, 4, True)
    psi = series_psi(g)
    assert psi.shape == (90, 3)
    C = g.psi6_acf(40)
    for r in range(3):
        want = oracle_mod.psi6_acf(psi[:, r], 40)
        assert np.abs(C[r] - want).max() <= 1e-12
        assert C[r, 0] == pytest.approx(1.0, abs=1e-15)
    tau = g.psi6_tau(1, 15)
    for r in range(3):
        want = oracle_mod.acf_tau(oracle_mod.psi6_acf(psi[:, r], 15), 1, 15)
        if np.isnan(want):
            assert np.isnan(tau[r])
        else:
            assert tau[r] == pytest.approx(want, rel=1e-9)
    from paper_1211_1645_gb300.hd import HD_ERR_ARG, HDError
    for bad in (lambda: g.psi6_acf(90), lambda: g.psi6_tau(5, 90), lambda: g.psi6_tau(6, 5)):
        with pytest.raises(HDError) as e:
            bad()
        assert e.value.status == HD_ERR_ARG
    g.close()


@pytest.mark.parametrize("form", ["fixed", "fp64"])
@pytest.mark.parametrize("bins", [1, 5, 16])
def test_field_matches_the_oracle(hd, oracle_mod, form, bins):
    N = 1000
    g = hd.HardDisks(N, 0.70, 0.12, 8, precision=form)
    o = oracle_mod.OracleChain(N, 0.70, 0.12, 8, form=form)
    g.sweep(25)
    o.sweep(25)
    f = g.psi6_field(bins)[0]
    loc, _ = o.psi6()
    geo = o.geometry()
    want = oracle_mod.psi6_field(o.positions(), loc, geo["L"], bins, LF=geo["LF"] if form == "fixed" else None)
    empty = np.isnan(want.real)
    assert np.array_equal(np.isnan(f.real), empty)
    assert np.abs(f[~empty] - want[~empty]).max() <= PSI_TOL[form]
    if bins == 1:  # one area: the mean over all disks, Psi_6
        glob, _ = g.psi6(want_local=False)
        assert abs(f[0, 0] - glob[0]) < 1e-12
    g.close()


def test_field_of_a_batch_and_argument_errors(hd, oracle_mod):
    g = hd.HardDisks([256, 400], [0.70, 0.60], [0.1, 0.1], [1, 2], precision="fixed")
    f = g.psi6_field(4)
    assert f.shape == (2, 4, 4)
    from paper_1211_1645_gb300.hd import HD_ERR_ARG, HDError
    with pytest.raises(HDError) as e:
        g.psi6_field(0)
    assert e.value.status == HD_ERR_ARG
    g.close()
