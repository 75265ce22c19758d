"""Pins of the oracle's MPMC chain (Sec. II.B) against facts that do not come
from the oracle itself: hard-core geometry, exact frame arithmetic and the
exact two-disk equilibrium law."""
import numpy as np
import pytest

from helpers import batch_se, min_image_d2, min_image_d2_fixed, to_fixed


@pytest.mark.parametrize("N,eta", [(256, 0.70), (1000, 0.55), (65536, 0.708), (4096, 0.72)])
def test_geometry(oracle_mod, N, eta):
    o = oracle_mod.OracleChain(N, eta, 0.1, 1, form="fp64")
    g = o.geometry()
    L = np.sqrt(N * np.pi / eta)  # Sec. II.A: eta = N pi sigma^2 / L^2
    assert g["L"] == pytest.approx(L, rel=1e-15)
    assert g["m"] % 2 == 0 and g["m"] >= 4
    assert g["w"] >= 2.0 and L / (g["m"] + 2) < 2.0  # largest even m with w >= 2 sigma


@pytest.mark.parametrize("form", ["fp64", "fixed"])
@pytest.mark.parametrize("N,eta,lattice,delta", [(256, 0.70, "square", 0.1), (256, 0.72, "triangular", 0.15),
                                                 (300, 0.60, "square", 0.3)])
def test_never_overlap(oracle_mod, form, N, eta, lattice, delta):
    """No accepted move may create an overlap; checked by brute force on
    global coordinates after every few sweeps."""
    o = oracle_mod.OracleChain(N, eta, delta, 11, form=form, lattice=lattice)
    g = o.geometry()
    for _ in range(20):
        o.sweep(5)
        xy = o.positions()
        if form == "fixed":
            r2 = min_image_d2_fixed(to_fixed(xy), g["LF"])
            assert r2.min() >= (1 << 50)
        else:
            assert min_image_d2(xy, g["L"]).min() >= 4.0 * (1 - 1e-12)
    att, acc = o.stats()
    assert 0 < acc < att


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_frame_consistency(oracle_mod, form):
    """Every disk sits inside its cell of the current shifted frame, and the
    frame reproduces the global positions."""
    o = oracle_mod.OracleChain(256, 0.70, 0.2, 5, form=form)
    o.sweep(37)
    g = o.geometry()
    cells, offs, shift = o.frame()
    assert cells.min() >= 0 and cells.max() < g["m"]
    assert offs.min() >= 0.0 and offs.max() < g["w"]
    assert (shift >= 0).all() and (shift < g["w"]).all()
    xy = (cells * g["w"] + offs + shift) % g["L"]
    d = xy - o.positions()
    d -= g["L"] * np.round(d / g["L"])
    assert np.abs(d).max() < 1e-12


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_zero_step_frame_invariance(oracle_mod, form):
    """With delta = 0 every trial is accepted and nothing moves: 30 grid
    shifts and rebuilds must leave the global positions unchanged (exactly in
    fixed point, up to FP64 rounding of the frame change otherwise)."""
    o = oracle_mod.OracleChain(256, 0.70, 0.0, 9, form=form, lattice="triangular")
    x0 = o.positions()
    o.sweep(30)
    att, acc = o.stats()
    assert att == acc > 0
    x1 = o.positions()
    if form == "fixed":
        assert np.array_equal(x0, x1)
    else:
        d = x1 - x0
        L = o.geometry()["L"]
        d -= L * np.round(d / L)
        assert np.abs(d).max() < 1e-12


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_attempts_one_per_occupied_cell(oracle_mod, form):
    """Each cell is active exactly once per sweep and an occupied cell makes
    n_t trials (Sec. II.B: a fixed number of trial moves per cell)."""
    o = oracle_mod.OracleChain(400, 0.65, 0.1, 2, form=form, nt=3)
    for _ in range(5):
        a0, _ = o.stats()
        o.sweep(1)
        a1, _ = o.stats()
        cells, _, _ = o.frame()  # cell membership does not change inside a sweep
        occupied = len({(int(c[0]), int(c[1])) for c in cells})
        assert a1 - a0 == 3 * occupied


def test_determinism_and_seed(oracle_mod):
    a = oracle_mod.OracleChain(256, 0.7, 0.1, 1, form="fp64")
    b = oracle_mod.OracleChain(256, 0.7, 0.1, 1, form="fp64")
    c = oracle_mod.OracleChain(256, 0.7, 0.1, 2, form="fp64")
    for o in (a, b, c):
        o.sweep(10)
    assert np.array_equal(a.positions(), b.positions())
    assert not np.array_equal(a.positions(), c.positions())


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_two_disk_separation_law(oracle_mod, form):
    """Two disks in a periodic 10 x 10 box: in equilibrium the minimum-image
    separation vector is uniform over the torus minus the excluded disk of
    radius 2 sigma, so P(r <= R) = (pi R^2 - 4 pi) / (V - 4 pi) for
    2 <= R <= L/2 (from the flat Boltzmann weight of Eq. 3).  A wrong overlap
    threshold, a biased proposal or a biased frame shift shows up here."""
    eta = 2 * np.pi / 100.0
    o = oracle_mod.OracleChain(2, eta, 1.0, 12345, form=form)
    g = o.geometry()
    L = g["L"]
    assert g["m"] == 4 and abs(L - 10.0) < 1e-6
    o.sweep(200)
    nsamp = 60000
    r = np.empty(nsamp)
    for t in range(nsamp):
        o.sweep(2)
        xy = o.positions()
        d = xy[1] - xy[0]
        d -= L * np.round(d / L)
        r[t] = np.hypot(d[0], d[1])
    assert r.min() >= 2.0 - 1e-12
    V = L * L
    for R in (2.5, 3.0, 3.5, 4.0, 4.5, 5.0):
        want = (np.pi * R * R - 4 * np.pi) / (V - 4 * np.pi)
        mean, se = batch_se(r <= R)
        assert abs(mean - want) < 5 * se + 1e-3, (R, mean, want, se)


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_eight_disks_against_rejection_sampling(oracle_mod, form):
    """Eight disks in a periodic 12 x 12 box (eta = 0.175) with 3-sigma cells
    (two disks share a cell about half of the time, capacity-9 geometry) and
    three trials per occupied cell: the chain's equilibrium distribution of
    collective coordinates (the smallest pair distance and disk 0's nearest-
    neighbour distance) must match exact samples of the uniform non-overlap
    measure (Eq. 3), drawn by rejection from independent uniform positions.
    This pins the stationary distribution with multi-occupied cells, their
    shuffles, repeated trials of one cell and the frame shifts together.
    (Any position-independent choice of the moving disk leaves that
    distribution unchanged: every single move satisfies detailed balance.)"""
    L, N = 12.0, 8
    eta = N * np.pi / (L * L)
    o = oracle_mod.OracleChain(N, eta, 0.8, 2024, form=form, nt=3, cell_min=3.0)
    geo = o.geometry()
    assert geo["m"] == 4 and geo["nt"] == 3 and abs(geo["L"] - L) < 1e-6
    iu = np.triu_indices(N, 1)

    def stats(xy):  # xy [..., N, 2] -> (min pair distance, disk 0's nearest neighbour)
        d = xy[..., :, None, :] - xy[..., None, :, :]
        d -= L * np.round(d / L)
        r = np.hypot(d[..., 0], d[..., 1])
        return r[..., iu[0], iu[1]].min(axis=-1), r[..., 0, 1:].min(axis=-1)

    o.sweep(500)
    nsamp = 25000
    mc = np.empty((nsamp, 2))
    multi = 0
    for t in range(nsamp):
        o.sweep(2)
        mc[t] = stats(o.positions())
        cells, _, _ = o.frame()
        multi += len({tuple(c) for c in cells}) < N
    assert multi > 0.3 * nsamp  # cells with two disks are common

    rng = np.random.default_rng(77)
    ref = []
    while sum(len(a) for a in ref) < 60000:
        xy = rng.uniform(0.0, L, (100000, N, 2))
        d = xy[:, :, None, :] - xy[:, None, :, :]
        d -= L * np.round(d / L)
        r = np.hypot(d[..., 0], d[..., 1])
        ok = r[:, iu[0], iu[1]].min(axis=1) >= 2.0
        ref.append(np.stack(stats(xy[ok]), axis=1))
    ref = np.concatenate(ref)
    for col, cuts in ((0, (2.1, 2.25, 2.5, 3.0)), (1, (2.5, 3.0, 3.5, 4.0))):
        for R in cuts:
            want = float(np.mean(ref[:, col] <= R))
            want_se = np.sqrt(want * (1 - want) / len(ref))
            mean, se = batch_se(mc[:, col] <= R)
            assert abs(mean - want) < 5 * np.hypot(se, want_se) + 2e-3, (col, R, mean, want, se)


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_openmp_sweep_is_the_same_chain(oracle_mod, form):
    """The all-cores sweep (each colour's cells shared out between threads)
    is bit-identical to the sequential oracle: positions and trial counts."""
    a = oracle_mod.OracleChain(4096, 0.70, 0.12, 5, form=form)
    b = oracle_mod.OracleChain(4096, 0.70, 0.12, 5, form=form)
    if not b.sweep_omp(1, 4):
        pytest.skip("no OpenMP in this compiler")
    a.sweep(1)
    for n in (6, 13):
        a.sweep(n)
        b.sweep_omp(n, 4)
        assert a.stats() == b.stats()
        assert np.array_equal(a.positions(), b.positions())
