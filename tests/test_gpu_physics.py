"""GPU tests of the chain's statistics: step-size tuning, and agreement of
the fixed-point and FP64 equations of state (different Markov chains of the
same ensemble) within three combined standard errors over independent
replicas."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import paper_1211_1645_gb300 as hd
    hd.load()
    return hd


@pytest.mark.parametrize("form,N", [("fixed", 65536), ("fp64", 16384)])
def test_tune_delta_reaches_target_acceptance(hd, form, N):
    """The N = 256^2, eta = 0.708 liquid is run with delta tuned to ~30%
    acceptance; after tuning the
    acceptance of later sweeps is within 0.03 of the target."""
    g = hd.HardDisks(N, 0.708, 0.1, 3, precision=form)
    g.sweep(100)
    d = g.tune_delta(0.30, sweeps_per_probe=20, probes=12)
    assert 0.0 < d[0] < g.geometry()["w"]
    a0, c0 = (int(x[0]) for x in g.stats())
    g.sweep(100)
    a1, c1 = (int(x[0]) for x in g.stats())
    assert abs((c1 - c0) / (a1 - a0) - 0.30) < 0.03


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_set_delta_matches_oracle(hd, oracle_mod, form):
    g = hd.HardDisks(1000, 0.65, 0.1, 5, precision=form)
    g.set_delta(0.2)
    o = oracle_mod.OracleChain(1000, 0.65, 0.2, 5, form=form)
    g.sweep(25)
    o.sweep(25)
    assert np.array_equal(g.positions(), o.positions())
    from paper_1211_1645_gb300.hd import HD_ERR_ARG, HDError
    with pytest.raises(HDError) as e:
        g.set_delta(10.0)  # beyond the cell side
    assert e.value.status == HD_ERR_ARG


def test_fixed_vs_fp64_equation_of_state(hd):
    """Eq. 4 pressure at eta = 0.716, N = 64^2, in both number forms (two
    different Markov chains of the same ensemble): sixteen independent
    replicas per form in one batch, 1.5 10^5 sweeps of equilibration from the
    square lattice, then 2 10^5 sweeps with the contact pressure every 1000.
    Errors are batch means over the independent replicas (the spread of the
    replica means).  Equilibration check: in each form the two halves of the
    production run agree within 3 standard errors.  The two forms' P* must
    agree within 3 combined standard errors."""
    R, N, eta = 16, 4096, 0.716
    equil, prod, every = 150_000, 200_000, 1000
    res = {}
    for form, seed0 in (("fixed", 100), ("fp64", 200)):
        g = hd.HardDisks([N] * R, [eta] * R, [0.1] * R, [seed0 + r for r in range(R)], precision=form)
        g.run(equil // every, every, False)
        g.series_reserve(prod // every + 8)
        g.run(prod // every, every, True)
        s = g.series()  # [step, replica, 4]
        etas = np.array([g.geometry(r)["eta"] for r in range(R)])
        pstar = s[:, :, 0] * 4.0 * etas / np.pi  # P* = beta P (2 sigma)^2
        g.close()
        T = pstar.shape[0]
        assert T == prod // every
        halves = [pstar[: T // 2].mean(axis=0), pstar[T // 2:].mean(axis=0)]
        h_se = [h.std(ddof=1) / np.sqrt(R) for h in halves]
        assert abs(halves[0].mean() - halves[1].mean()) < 3.0 * np.hypot(*h_se), (form, halves)
        means = pstar.mean(axis=0)
        res[form] = (means.mean(), means.std(ddof=1) / np.sqrt(R))
    (mf, sf), (md, sd) = res["fixed"], res["fp64"]
    print(f"P* at eta = 0.716, N = 64^2: fixed point {mf:.4f} +- {sf:.4f}, FP64 {md:.4f} +- {sd:.4f}, "
          f"difference {(mf - md) / np.hypot(sf, sd):+.2f} combined SE")
    assert abs(mf - md) < 3.0 * np.hypot(sf, sd), res


def test_autotuner_picks_a_valid_fast_configuration(hd):
    from paper_1211_1645_gb300.tune import autotune
    best, table = autotune(65536, 0.708, 0.1, cell_mins=(2.0, 2.4), block_threads=(128, 256),
                           threads_per_cell=(1, 2), strips=(1, 16), sweeps=20, steps=2)
    assert best is not None and len(table) >= 8
    assert best["trial_moves_per_s"] == max(r["trial_moves_per_s"] for r in table)
    assert best["cell_min"] in (2.0, 2.4) and best["sweep_kernel"] in ("split", "fused")
    assert {r["threads_per_cell"] for r in table} == {1, 2}
    # strips only on the split one-thread pass, where the step graph then has that many branches
    assert {(r["strips"], r["graph_branches"]) for r in table if r["sweep_kernel"] == "split"
            and r["threads_per_cell"] == 1} == {(1, 1), (16, 16)}


def test_autotuner_per_replica_choice_runs_the_same_chains(hd, oracle_mod):
    """autotune_replicas picks a cell side per state point and the batch's
    launch shape; a batch built from its choice runs each replica's own chain
    (as the oracle with that cell side)."""
    from paper_1211_1645_gb300.tune import autotune_replicas
    Ns, etas = [32 ** 2, 24 ** 2, 32 ** 2], [0.70, 0.60, 0.72]
    choice, table = autotune_replicas(Ns, etas, 0.1, seed=5, cell_mins=(2.0, 2.6), block_threads=(64, 128),
                                      threads_per_cell=(1, 2), sweeps=10, steps=2)
    assert choice is not None and len(choice["cell_min"]) == 3 and len(table) in (4, 8)
    assert choice["trial_moves_per_s"] == max(r["trial_moves_per_s"] for r in table)
    g = hd.HardDisks(Ns, etas, [0.1] * 3, [5, 6, 7], precision="fixed", cell_min=choice["cell_min"],
                     block_threads=choice["block_threads"], threads_per_cell=choice["threads_per_cell"])
    g.run(2, 10, False)
    xy = g.positions()
    off = 0
    for r, (n, e, cm) in enumerate(zip(Ns, etas, choice["cell_min"])):
        o = oracle_mod.OracleChain(n, e, 0.1, 5 + r, form="fixed", cell_min=cm)
        o.sweep(20)
        assert np.array_equal(xy[off:off + n], o.positions())
        off += n
    g.close()


@pytest.mark.slow
@pytest.mark.skipif(__import__("os").environ.get("HD_SLOW") != "1",
                    reason="about two minutes of GPU time: set HD_SLOW=1")
def test_table1_mpmc_pressure_anchor(hd):
    """Table I: N = 256^2 at eta = 0.698, MPMC P* = 9.17078 +- 4.5e-5 (8 runs
    of 6e13 displacements).  Eight fixed-point replicas from the square
    lattice, 10^6 sweeps of equilibration (Table II's tau at N = 512^2 is
    8e5 displacements per disk), then 2 10^6 sweeps with the contact pressure
    (100 bins of 10^-3 sigma, the paper's shell) every 1000 sweeps.  The
    replica means must agree with the paper within three combined standard
    errors (ours from the spread of the eight replica means)."""
    import os
    R, N, eta = 8, 256 * 256, 0.698
    equil = int(os.environ.get("HD_SLOW_EQUIL", "1000000"))
    prod = int(os.environ.get("HD_SLOW_PROD", "2000000"))
    every = 1000
    g = hd.HardDisks([N] * R, [eta] * R, [0.1] * R, [101 + r for r in range(R)], precision="fixed",
                     hist_bins=100, hist_dr=1e-3)
    g.run(equil // every, every, False)
    g.series_reserve(prod // every + 8)
    g.run(prod // every, every, True)
    s = g.series()  # [T, R, 4]: beta P / rho first
    etas = np.array([g.geometry(r)["eta"] for r in range(R)])
    pstar = s[:, :, 0] * 4.0 * etas / np.pi  # P* = beta P (2 sigma)^2 = (beta P / rho) 4 eta / pi
    means = pstar.mean(axis=0)
    se = means.std(ddof=1) / np.sqrt(R)
    want, want_se = 9.17078, 4.5e-5
    print(f"P* = {means.mean():.5f} +- {se:.5f} (replica means {np.round(means, 4).tolist()}), paper {want} +- {want_se}")
    assert abs(means.mean() - want) < 3.0 * np.hypot(se, want_se)
    g.close()


@pytest.mark.slow
@pytest.mark.skipif(__import__("os").environ.get("HD_SLOW") != "1",
                    reason="a few minutes of GPU time: set HD_SLOW=1")
def test_fixed_vs_fp64_equation_of_state_long(hd):
    """The fixed-point chain's pressure at eta = 0.716 (N = 128^2) must agree
    with the FP64 chain's within three combined standard errors: eight
    independent replicas per form, 10^6 sweeps of equilibration from the
    square lattice, then 10^6 sweeps with the contact pressure every 1000
    sweeps.  The two forms are different Markov chains of the same ensemble,
    so the comparison is statistical."""
    import os
    R, N, eta = 8, 128 * 128, 0.716
    equil = int(os.environ.get("HD_SLOW_EQUIL", "1000000"))
    prod = int(os.environ.get("HD_SLOW_PROD", "1000000"))
    every = 1000
    out = {}
    for form, seed0 in (("fixed", 300), ("fp64", 400)):
        g = hd.HardDisks([N] * R, [eta] * R, [0.1] * R, [seed0 + r for r in range(R)], precision=form)
        g.run(equil // every, every, False)
        g.series_reserve(prod // every + 8)
        g.run(prod // every, every, True)
        s = g.series()
        etas = np.array([g.geometry(r)["eta"] for r in range(R)])
        means = (s[:, :, 0] * 4.0 * etas / np.pi).mean(axis=0)  # P* per replica
        out[form] = (means.mean(), means.std(ddof=1) / np.sqrt(R))
        g.close()
    (mf, sf), (md, sd) = out["fixed"], out["fp64"]
    print(f"P* fixed {mf:.5f} +- {sf:.5f}, FP64 {md:.5f} +- {sd:.5f}, difference {(mf - md) / np.hypot(sf, sd):.2f} SE")
    assert abs(mf - md) < 3.0 * np.hypot(sf, sd)


@pytest.mark.slow
@pytest.mark.skipif(__import__("os").environ.get("HD_SLOW") != "1",
                    reason="about ten minutes of GPU time: set HD_SLOW=1")
def test_table2_psi6_correlation_time(hd):
    """Table II: at N = 512^2, eta = 0.698 the Psi_6 correlation time of MPMC
    is 8e5 displacements per disk.  Four fixed-point replicas from the square
    lattice, delta tuned to 30% acceptance (the paper leaves MPMC's step to
    'optimal internal parameters'), 2e6 sweeps of equilibration, then 1e7
    sweeps with Psi_6 recorded every 1000.  tau comes from the Eq. 9
    autocorrelation, averaged over the replicas, fitted (ln Re C against the
    lag) where 0.05 < Re C < 0.5, and is converted to displacements per disk
    with the chain's attempts per disk per sweep.  The step size enters tau,
    so the check is loose: within a factor of four of the paper's value."""
    import os
    import time as _time
    R, N, eta = 4, 512 * 512, 0.698
    equil = int(os.environ.get("HD_SLOW_EQUIL", "2000000"))
    prod = int(os.environ.get("HD_SLOW_PROD", "10000000"))
    every = 1000
    g = hd.HardDisks([N] * R, [eta] * R, [0.1] * R, [501 + r for r in range(R)], precision="fixed")
    g.run(200, 100, False)
    delta = g.tune_delta(0.3, 50, 20)
    g.run(equil // every, every, False)
    a0, c0 = (x.sum() for x in g.stats())
    g.series_reserve(prod // every + 8)
    t0 = _time.perf_counter()
    g.run(prod // every, every, True)
    a1, c1 = (x.sum() for x in g.stats())  # synchronises
    wall = _time.perf_counter() - t0
    disp_per_sweep = float(a1 - a0) / (R * N * (prod // every) * every)  # attempts per disk per sweep
    T = prod // every
    C = g.psi6_acf(T // 3).real.mean(axis=0)
    lags = np.arange(C.size)
    sel = (C > 0.05) & (C < 0.5)
    assert sel.sum() >= 5, f"no exponential window: C = {np.round(C[:50], 3).tolist()}"
    slope = np.polyfit(lags[sel], np.log(C[sel]), 1)[0]
    tau_steps = -1.0 / slope
    tau_lib = g.psi6_tau(int(lags[sel][0]), int(lags[sel][-1]))
    tau_disp = tau_steps * every * disp_per_sweep
    s_per_tau = wall / (prod / every) * tau_steps
    print(f"delta {np.round(delta, 4).tolist()}, acceptance {float(c1 - c0) / float(a1 - a0):.3f}, "
          f"tau = {tau_steps:.0f} recorded steps = {tau_disp:.3g} displacements per disk "
          f"(per replica {np.round(tau_lib * every * disp_per_sweep, -3).tolist()}), paper 8e5; "
          f"{s_per_tau:.1f} s of GPU time per tau for the four replicas")
    assert 8e5 / 4 < tau_disp < 8e5 * 4
    g.close()


@pytest.mark.parametrize("layout", ["one", "strips", "branches"])
@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_set_delta_reaches_captured_steps(hd, form, layout):
    """One-replica launches (a single replica, its strips, or each replica's
    branch of a batch) take the replica's constants by value, so a changed
    delta must reach the graph-captured steps too: graph steps with a delta
    change in between equal direct sweeps with the same change."""
    if layout == "branches":
        args = ([1000, 576, 784], [0.65, 0.66, 0.64], [0.1] * 3, [6, 7, 8])
        new_delta = [0.25, 0.2, 0.15]
    else:
        args = (1000, 0.65, 0.1, 6)
        new_delta = 0.25
    kw = {"strips": 3} if layout == "strips" else {}
    a = hd.HardDisks(*args, precision=form, **kw)
    b = hd.HardDisks(*args, precision=form)
    assert a.geometry()["graph_branches"] == {"one": 1, "strips": 3, "branches": 3}[layout]
    a.run(1, 7, False)
    b.sweep(7)
    a.set_delta(new_delta)
    b.set_delta(new_delta)
    a.run(2, 7, False)
    b.sweep(14)
    assert np.array_equal(a.positions(), b.positions())
    assert [x.tolist() for x in a.stats()] == [x.tolist() for x in b.stats()]
    a.close()
    b.close()
