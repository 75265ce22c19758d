"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bar: positions, trial counts and histogram counts bit-exact (FP64 with no FMA
on both sides, and the fixed-point form); pressure within 1e-12 relative to
max(1, |value|) (PRESSURE_TOL);
every psi_j and the global Psi_6 bit-exact in both forms (the same operations
in the same order per disk, and the global sum exactly rounded on both sides
before the division by N), which meets the 1e-12 relative bar with no
rounding allowance at all.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# Pressure bar: 1e-12 relative to max(1, |x|) for g(2 sigma+) and for
# beta P / rho = 1 + 2 eta g(2 sigma+).  The GPU fits by Householder QR, the
# oracle by numpy's least squares, so the two agree to rounding; where the
# extrapolated g is near -1 / (2 eta) (a sparse histogram just after the
# lattice start), beta P / rho is a cancellation and only the unit scale of
# its leading 1 is meaningful.
PRESSURE_TOL = 1e-12


CASES = {
    "square_N256": dict(N=256, eta=0.70, delta=0.1, seed=1),
    "ragged_N1000": dict(N=1000, eta=0.55, delta=0.25, seed=7),
    "triangular": dict(N=256, eta=0.72, delta=0.15, seed=3, lattice="triangular"),
    "three_trials": dict(N=400, eta=0.60, delta=0.2, seed=5, nt=3),
    "two_trials_wide_cells": dict(N=1000, eta=0.716, delta=0.1, seed=6, cell_min=2.2),
    "cap9_cells": dict(N=300, eta=0.50, delta=0.4, seed=9, cell_min=3.0),
    "two_disks": dict(N=2, eta=2 * math.pi / 100, delta=1.0, seed=4),
    # square lattice 0.007 sigma from contact with tiny steps: many pairs land
    # near contact, where the FP64 form's float pre-test hands over to FP64
    "near_contact_dense": dict(N=1024, eta=0.78, delta=0.004, seed=12),
}


@pytest.fixture(scope="module")
def hd():
    import paper_1211_1645_gb300 as hd
    hd.load()
    return hd


def make_pair(hd, oracle_mod, form, N, eta, delta, seed, lattice="square", nt=0, cell_min=2.0, K=50, dr=1e-3,
              kernel="split"):
    """kernel: "split", "tma", "fused", or "split-g<G>" for the split pass with
    G threads per active cell."""
    tpc = 1
    if kernel.startswith("split-g"):
        kernel, tpc = "split", int(kernel[len("split-g"):])
    g = hd.HardDisks(N, eta, delta, seed, precision=form, lattice=lattice, trials_per_cell=nt, cell_min=cell_min,
                     hist_bins=K, hist_dr=dr, sweep_kernel=kernel, threads_per_cell=tpc,
                     block_threads=64 if tpc == 8 else 128)
    o = oracle_mod.OracleChain(N, eta, delta, seed, form=form, lattice=lattice, nt=nt, cell_min=cell_min)
    return g, o


def assert_same_state(g, o):
    att, acc = g.stats()
    assert (int(att[0]), int(acc[0])) == o.stats()
    assert np.array_equal(g.positions(), o.positions())


@pytest.mark.parametrize("kernel", ["fused", "split", "tma", "persistent", "split-g2", "split-g4", "split-g8"])
@pytest.mark.parametrize("form", ["fp64", "fixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_chain_bit_exact(hd, oracle_mod, form, case, kernel):
    """Every sweep kernel: one launch per sweep with shared-memory tiles; a
    rebuild launch plus four colour-pass launches (one thread per active
    cell, bulk-copy staging, or G = 2, 4, 8 threads per cell with a warp
    ballot over the overlap tests); one persistent launch per call of up to
    256 sweeps (a wavefront of band work items)."""
    g, o = make_pair(hd, oracle_mod, form, kernel=kernel, **CASES[case])
    geo, ogeo = g.geometry(), o.geometry()
    assert geo["m"] == ogeo["m"] and geo["L"] == ogeo["L"] and geo["trials_per_cell"] == ogeo["nt"]
    assert_same_state(g, o)  # the initial lattice
    for n in (1, 9, 90):
        g.sweep(n)
        o.sweep(n)
        assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("kernel", ["fused", "split", "tma", "persistent"])
@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_chunk_boundary(hd, oracle_mod, form, kernel):
    """More sweeps in one call than one draw table holds (256)."""
    g, o = make_pair(hd, oracle_mod, form, 256, 0.70, 0.1, 21, kernel=kernel)
    g.sweep(300)
    o.sweep(300)
    assert_same_state(g, o)
    g.sweep(0)
    assert_same_state(g, o)


@pytest.mark.parametrize("form", ["fp64", "fixed"])
@pytest.mark.parametrize("K,dr", [(50, 1e-3), (100, 1e-3), (37, 0.004)])
def test_pressure(hd, oracle_mod, form, K, dr):
    g, o = make_pair(hd, oracle_mod, form, 1000, 0.70, 0.1, 17, K=K, dr=dr)
    for n in (0, 25):
        g.sweep(n)
        o.sweep(n)
        bp, g0, hist = g.pressure()
        want_hist = o.histogram(K, dr)
        assert np.array_equal(hist[0], want_hist)
        want = oracle_mod.contact_pressure(want_hist, 1000, o.geometry()["L"], o.realised_dr(dr))
        assert abs(bp[0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
        assert abs(g0[0] - want["g0"]) <= PRESSURE_TOL * max(1.0, abs(want["g0"]))


@pytest.mark.parametrize("form", ["fp64", "fixed"])
@pytest.mark.parametrize("case", ["square_N256", "ragged_N1000", "cap9_cells"])
def test_psi6(hd, oracle_mod, form, case):
    g, o = make_pair(hd, oracle_mod, form, **CASES[case])
    g.sweep(40)
    o.sweep(40)
    glob, loc = g.psi6()
    rloc, rglob = o.psi6()
    assert np.array_equal(loc, rloc)
    assert glob[0] == rglob
    glob2, none = g.psi6(want_local=False)
    assert none is None and glob2[0] == glob[0]


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_psi6_low_density_ring_search(hd, oracle_mod, form):
    """At eta = 0.15 the sixth neighbour often lies beyond the first 5 x 5 cells."""
    g, o = make_pair(hd, oracle_mod, form, 256, 0.15, 1.0, 8)
    g.sweep(50)
    o.sweep(50)
    glob, loc = g.psi6()
    rloc, rglob = o.psi6()
    assert np.array_equal(loc, rloc)
    assert glob[0] == rglob


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_set_positions_roundtrip(hd, oracle_mod, form):
    g, o = make_pair(hd, oracle_mod, form, 400, 0.65, 0.15, 2)
    rng = np.random.default_rng(0)
    g.sweep(30)
    o.sweep(30)
    xy = o.positions() + rng.integers(-2, 3, size=(400, 2)) * o.geometry()["L"]  # periodic images
    g.set_positions(xy)
    o.set_positions(xy)
    assert np.array_equal(g.positions(), o.positions())
    g.sweep(7)
    o.sweep(7)
    assert np.array_equal(g.positions(), o.positions())


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_batched_replicas(hd, oracle_mod, form):
    """Independent chains of uneven N and eta in one context (the
    equation-of-state scan as one batch): each equals its own oracle chain."""
    Ns = [16 ** 2, 24 ** 2, 32 ** 2, 20 ** 2, 17 ** 2]
    etas = [0.700, 0.701, 0.702, 0.703, 0.704]
    deltas = [0.1, 0.12, 0.09, 0.11, 0.1]
    seeds = [101, 102, 103, 104, 105]
    g = hd.HardDisks(Ns, etas, deltas, seeds, precision=form)
    os_ = [oracle_mod.OracleChain(n, e, d, s, form=form) for n, e, d, s in zip(Ns, etas, deltas, seeds)]
    g.sweep(60)
    for o in os_:
        o.sweep(60)
    att, acc = g.stats()
    xy = g.positions()
    off = 0
    bp, g0, hist = g.pressure()
    glob, loc = g.psi6()
    for r, o in enumerate(os_):
        assert (int(att[r]), int(acc[r])) == o.stats()
        assert np.array_equal(xy[off:off + Ns[r]], o.positions())
        h = o.histogram(50, 1e-3)
        assert np.array_equal(hist[r], h)
        want = oracle_mod.contact_pressure(h, Ns[r], o.geometry()["L"], o.realised_dr(1e-3))
        assert abs(bp[r] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
        rloc, rglob = o.psi6()
        assert np.array_equal(loc[off:off + Ns[r]], rloc)
        assert glob[r] == rglob
        off += Ns[r]


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_full_size_N65536_liquid(hd, oracle_mod, form):
    """N = 256^2 at eta = 0.708 (liquid side), whole state compared."""
    g, o = make_pair(hd, oracle_mod, form, 65536, 0.708, 0.1, 2)
    g.sweep(20)
    o.sweep(20)
    assert_same_state(g, o)
    bp, _, hist = g.pressure()
    assert np.array_equal(hist[0], o.histogram(50, 1e-3))


@pytest.mark.parametrize("kernel", ["fused", "split", "tma", "persistent"])
@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_full_size_N1048576_coexistence(hd, oracle_mod, form, kernel):
    """N = 1024^2 at eta = 0.716 (coexistence), the benchmark workload: whole
    state, histogram and every psi_j compared after three sweeps."""
    N = 1024 * 1024
    g, o = make_pair(hd, oracle_mod, form, N, 0.716, 0.1, 1, kernel=kernel)
    g.sweep(3)
    o.sweep(3)
    assert_same_state(g, o)
    bp, _, hist = g.pressure()
    want_hist = o.histogram(50, 1e-3)
    assert np.array_equal(hist[0], want_hist)
    want = oracle_mod.contact_pressure(want_hist, N, o.geometry()["L"], o.realised_dr(1e-3))
    assert abs(bp[0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
    glob, loc = g.psi6()
    rloc, rglob = o.psi6()
    assert np.array_equal(loc, rloc)
    assert glob[0] == rglob


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_full_size_bench_step(hd, oracle_mod, form):
    """The benchmark's own launch path at its size: N = 1024^2, eta = 0.716,
    seed 1, one graph-captured step of 100 sweeps and a device-side
    measurement on a library stream of the caller's (hd_run, as bench.py
    times it); series entry, trial counts and every position against the
    oracle after the same 100 sweeps."""
    import torch
    N = 1024 * 1024
    g, o = make_pair(hd, oracle_mod, form, N, 0.716, 0.1, 1)
    s = torch.cuda.Stream()
    g.set_stream(s.cuda_stream)
    g.series_reserve(4)
    g.run(1, 100, measure=True)
    ser = g.series()
    o.sweep(100)
    want = oracle_mod.contact_pressure(o.histogram(50, 1e-3), N, o.geometry()["L"], o.realised_dr(1e-3))
    _, rglob = o.psi6()
    assert abs(ser[0, 0, 0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
    assert complex(ser[0, 0, 2], ser[0, 0, 3]) == rglob
    assert_same_state(g, o)


def test_full_size_N4194304_shifted_rows(hd, oracle_mod):
    """N = 2048^2 at eta = 0.720 from the shifted-row lattice, fixed point."""
    N = 2048 * 2048
    g, o = make_pair(hd, oracle_mod, "fixed", N, 0.720, 0.1, 5, lattice="triangular")
    g.sweep(2)
    o.sweep(2)
    assert_same_state(g, o)
    _, _, hist = g.pressure()
    assert np.array_equal(hist[0], o.histogram(50, 1e-3))


def test_largest_size_N16777216(hd, oracle_mod):
    """N = 4096^2 at eta = 0.716, fixed point: the largest N of the
    allocation-free Psi_6 mean (4096 blocks of 4096 values) and 16x the
    benchmark.  Whole state, histogram and every psi_j after one sweep, and
    the allocation-free mean of the library's own psi_j field at exactly its
    size limit."""
    import ctypes
    import torch
    N = 4096 * 4096
    g, o = make_pair(hd, oracle_mod, "fixed", N, 0.716, 0.1, 11)
    g.sweep(1)
    o.sweep(1)
    assert_same_state(g, o)
    _, _, hist = g.pressure()
    assert np.array_equal(hist[0], o.histogram(50, 1e-3))
    glob, loc = g.psi6()
    rloc, rglob = o.psi6()
    assert np.array_equal(loc, rloc)
    assert glob[0] == rglob
    del o, rloc
    field = torch.from_numpy(np.stack([loc.real, loc.imag], 1).copy()).to("cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    lib = hd.load()
    st = lib.hd_psi6_mean_noalloc(ctypes.c_void_p(field.data_ptr()), ctypes.c_int64(N),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    torch.cuda.synchronize()
    assert st == 0
    got = out.cpu().numpy()
    assert complex(got[0], got[1]) == glob[0]
    g.close()


def test_reach_error_is_reported_and_recoverable(hd, oracle_mod):
    from paper_1211_1645_gb300.hd import HD_ERR_REACH, HDError
    g = hd.HardDisks(2, 2 * math.pi / 100, 1.0, 4, hist_bins=500, hist_dr=0.01)
    with pytest.raises(HDError) as e:
        g.pressure()
    assert e.value.status == HD_ERR_REACH
    g.sweep(5)  # still usable
    assert g.stats()[0][0] > 0


def test_psi6_reach_error(hd):
    from paper_1211_1645_gb300.hd import HD_ERR_REACH, HDError
    N, L = 8, 40.0
    g = hd.HardDisks(N, N * math.pi / L ** 2, 0.1, 1)
    # rows 10 apart in x and 20 in y: the sixth neighbour (22.4 sigma) lies beyond
    # the widest stencil a 40-sigma box allows (9 rings of 2-sigma cells)
    xy = np.array([[5 + 10 * (k % 4), 5 + 20 * (k // 4)] for k in range(N)], dtype=np.float64)
    g.set_positions(xy)
    with pytest.raises(HDError) as e:
        g.psi6()
    assert e.value.status == HD_ERR_REACH
    g.sweep(1)


def test_overflow_rejected_on_set_positions(hd):
    from paper_1211_1645_gb300.hd import HD_ERR_OVERFLOW, HDError
    g = hd.HardDisks(256, 0.7, 0.1, 1)
    xy = g.positions()
    xy[:5] = [[1.0, 1.0], [1.1, 1.0], [1.2, 1.0], [1.3, 1.0], [1.4, 1.0]]  # five disks in one cell
    with pytest.raises(HDError) as e:
        g.set_positions(xy)
    assert e.value.status == HD_ERR_OVERFLOW


@pytest.mark.parametrize("kernel", ["split", "fused", "tma", "persistent"])
@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_graph_engine_series(hd, oracle_mod, form, kernel):
    """hd_run: graph-captured steps of 7 sweeps (odd, so both buffer parities
    are captured) with a device-side measurement per step; the series must
    equal the oracle's pressure and Psi_6 after each step, and the chain must
    continue exactly."""
    g, o = make_pair(hd, oracle_mod, form, 400, 0.70, 0.1, 31, kernel=kernel)
    g.run(3, 7, measure=True)
    ser = g.series()
    assert ser.shape == (3, 1, 4)
    L = o.geometry()["L"]
    for k in range(3):
        o.sweep(7)
        h = o.histogram(50, 1e-3)
        want = oracle_mod.contact_pressure(h, 400, L, o.realised_dr(1e-3))
        _, rglob = o.psi6()
        assert abs(ser[k, 0, 0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
        assert abs(ser[k, 0, 1] - want["g0"]) <= PRESSURE_TOL * max(1.0, abs(want["g0"]))
        assert complex(ser[k, 0, 2], ser[k, 0, 3]) == rglob
    assert_same_state(g, o)
    g.run(2, 7, measure=False)
    o.sweep(14)
    assert_same_state(g, o)
    assert g.series().shape[0] == 3
    g.series_clear()
    assert g.series().shape[0] == 0


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_graph_engine_batched(hd, oracle_mod, form):
    Ns = [20 ** 2, 16 ** 2, 24 ** 2]
    etas = [0.70, 0.71, 0.705]
    g = hd.HardDisks(Ns, etas, [0.1] * 3, [7, 8, 9], precision=form)
    os_ = [oracle_mod.OracleChain(n, e, 0.1, s, form=form) for n, e, s in zip(Ns, etas, [7, 8, 9])]
    g.run(2, 10, measure=True)
    ser = g.series()
    assert ser.shape == (2, 3, 4)
    for k in range(2):
        for r, o in enumerate(os_):
            o.sweep(10)
            want = oracle_mod.contact_pressure(o.histogram(50, 1e-3), Ns[r], o.geometry()["L"], o.realised_dr(1e-3))
            assert abs(ser[k, r, 0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
            _, rglob = o.psi6()
            assert complex(ser[k, r, 2], ser[k, r, 3]) == rglob
    xy = g.positions()
    off = 0
    for r, o in enumerate(os_):
        assert np.array_equal(xy[off:off + Ns[r]], o.positions())
        off += Ns[r]


@pytest.mark.parametrize("kernel", ["split", "fused", "tma", "persistent"])
@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_checkpoint_resume_bit_exact(hd, oracle_mod, form, kernel):
    """A chain checkpointed after 40 sweeps and restored into a fresh context
    continues exactly as the uninterrupted chain (and as the oracle)."""
    g, o = make_pair(hd, oracle_mod, form, 1000, 0.70, 0.12, 77, kernel=kernel)
    g.sweep(40)
    blob = g.checkpoint()
    g.sweep(30)
    o.sweep(70)
    g2 = hd.HardDisks(1000, 0.70, 0.12, 77, precision=form, sweep_kernel=kernel)
    g2.restore(blob)
    g2.sweep(30)
    assert np.array_equal(g2.positions(), g.positions())
    assert [int(x[0]) for x in g2.stats()] == [int(x[0]) for x in g.stats()]
    assert_same_state(g2, o)
    assert g2.geometry()["sweeps"] == 70


def test_restore_rejects_other_geometry(hd):
    from paper_1211_1645_gb300.hd import HD_ERR_ARG, HDError
    g = hd.HardDisks(1000, 0.70, 0.12, 77, precision="fixed")
    blob = g.checkpoint()
    other = hd.HardDisks(1000, 0.70, 0.12, 78, precision="fixed")  # different seed
    with pytest.raises(HDError) as e:
        other.restore(blob)
    assert e.value.status == HD_ERR_ARG
    with pytest.raises(HDError):
        g.restore(blob[:100])


@pytest.mark.parametrize("threads", [32, 64, 256])
@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_tma_pass_block_sizes(hd, oracle_mod, form, threads):
    """The bulk-copy pass stages half-row segments whose width follows the
    block size: one segment per half-row (m/2 <= threads), several, and
    32-cell segments that wrap at both row ends; capacity-9 cells too."""
    for N, eta, cell_min in ((1000, 0.70, 2.0), (4096, 0.60, 3.0)):
        g = hd.HardDisks(N, eta, 0.15, 9, precision=form, sweep_kernel="tma", block_threads=threads,
                         cell_min=cell_min)
        o = oracle_mod.OracleChain(N, eta, 0.15, 9, form=form, cell_min=cell_min)
        for n in (1, 7, 24):
            g.sweep(n)
            o.sweep(n)
            assert_same_state(g, o)
        g.close()


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_profiled_graph_and_kept_local_field(hd, oracle_mod, form):
    """hd_run while profiling (a timing event around every kernel node of the
    step graph) runs the same chain, and times every launch; measure == 2
    keeps each measurement's psi_j field on the device, equal to the
    oracle's."""
    import torch
    g, o = make_pair(hd, oracle_mod, form, 1000, 0.70, 0.1, 41)
    g.profile(True)
    g.run(2, 5, measure=2)
    kt = g.kernel_times()
    g.profile(False)
    assert kt["pass"][1] == 2 * 5 * 4 and kt["rebuild"][1] == 2 * 5 and kt["psi6"][1] == 2
    assert all(ms > 0 for ms, n in kt.values() if n)
    o.sweep(10)
    assert_same_state(g, o)
    field = torch.empty(2 * 1000, dtype=torch.float64, device="cuda")
    g.psi6_local_device(field.data_ptr())
    torch.cuda.synchronize()
    f = field.cpu().numpy().reshape(-1, 2)
    rloc, rglob = o.psi6()
    assert np.array_equal(f[:, 0] + 1j * f[:, 1], rloc)
    ser = g.series()
    assert complex(ser[-1, 0, 2], ser[-1, 0, 3]) == rglob
    g.run(1, 5, measure=True)  # the unprofiled graph of the same step
    o.sweep(5)
    assert_same_state(g, o)


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_batched_replicas_per_replica_cell_sides(hd, oracle_mod, form):
    """Replicas with their own minimum cell sides (as the autotuner picks them
    per state point) in one context: each equals its own oracle chain with
    that cell side (trials per occupied cell 1, 2, 2 and 3, capacity-9
    cells), also with two threads per active cell."""
    Ns = [24 ** 2, 20 ** 2, 32 ** 2, 17 ** 2]
    etas = [0.70, 0.71, 0.705, 0.60]
    cms = [2.0, 2.4, 2.2, 3.0]
    seeds = [61, 62, 63, 64]
    for tpc in (1, 2):
        g = hd.HardDisks(Ns, etas, [0.1] * 4, seeds, precision=form, cell_min=cms, threads_per_cell=tpc)
        os_ = [oracle_mod.OracleChain(n, e, 0.1, sd, form=form, cell_min=cm) for n, e, sd, cm in zip(Ns, etas, seeds, cms)]
        for r, o in enumerate(os_):
            geo = g.geometry(r)
            assert geo["m"] == o.geometry()["m"] and geo["w"] >= cms[r]
        assert g.geometry(0)["w"] < 2.4 and g.geometry(3)["trials_per_cell"] == 3
        g.run(3, 10, measure=True)
        for o in os_:
            o.sweep(30)
        att, acc = g.stats()
        xy = g.positions()
        ser = g.series()
        off = 0
        for r, o in enumerate(os_):
            assert (int(att[r]), int(acc[r])) == o.stats()
            assert np.array_equal(xy[off:off + Ns[r]], o.positions())
            _, rglob = o.psi6()
            assert complex(ser[-1, r, 2], ser[-1, r, 3]) == rglob
            off += Ns[r]
        g.close()


def test_persistent_batched_replicas(hd, oracle_mod):
    """The persistent sweep over replicas of uneven N (their bands interleave
    in each phase), graph-captured steps with measurement, against each
    replica's oracle chain."""
    for form in ("fixed", "fp64"):
        Ns = [16 ** 2, 24 ** 2, 32 ** 2, 20 ** 2, 17 ** 2]
        etas = [0.700, 0.701, 0.702, 0.703, 0.704]
        seeds = [101, 102, 103, 104, 105]
        g = hd.HardDisks(Ns, etas, [0.1] * 5, seeds, precision=form, sweep_kernel="persistent")
        os_ = [oracle_mod.OracleChain(n, e, 0.1, sd, form=form) for n, e, sd in zip(Ns, etas, seeds)]
        g.run(3, 9, measure=True)
        g.sweep(5)
        for o in os_:
            o.sweep(32)
        att, acc = g.stats()
        xy = g.positions()
        off = 0
        for r, o in enumerate(os_):
            assert (int(att[r]), int(acc[r])) == o.stats()
            assert np.array_equal(xy[off:off + Ns[r]], o.positions())
            off += Ns[r]
        g.close()


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_config1_full_run(hd, oracle_mod, form):
    """The first configuration as specified: N = 256 on a 16 x 16 square
    lattice at eta = 0.70, delta = 0.1 sigma, seed 1, 10,000 sweeps through
    the graph engine with the contact pressure (50 bins of 1e-3 sigma) and the
    global Psi_6 recorded every 100 sweeps; every one of the 100 recorded
    entries against the oracle after the same sweeps, and the acceptance rate
    and final state."""
    g, o = make_pair(hd, oracle_mod, form, 256, 0.70, 0.1, 1)
    g.series_reserve(128)
    g.run(100, 100, measure=True)
    ser = g.series()
    assert ser.shape == (100, 1, 4)
    L = o.geometry()["L"]
    for k in range(100):
        o.sweep(100)
        want = oracle_mod.contact_pressure(o.histogram(50, 1e-3), 256, L, o.realised_dr(1e-3))
        _, rglob = o.psi6()
        assert abs(ser[k, 0, 0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
        assert complex(ser[k, 0, 2], ser[k, 0, 3]) == rglob
    assert_same_state(g, o)
    att, acc = g.stats()
    assert 0.3 < int(acc[0]) / int(att[0]) < 0.9


@pytest.mark.parametrize("lattice", ["square", "triangular"])
@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_psi6_on_the_start_lattice(hd, oracle_mod, form, lattice):
    """The untouched start lattice, where neighbour distances tie everywhere:
    the six-neighbour list's (r^2, id) order decides psi_j, on the GPU as in
    the oracle (square: two of the four tied diagonals by smaller id)."""
    g, o = make_pair(hd, oracle_mod, form, 1024, 0.60, 0.1, 3, lattice=lattice)
    glob, loc = g.psi6()
    rloc, rglob = o.psi6()
    assert np.array_equal(loc, rloc)
    assert glob[0] == rglob
    g.close()


STRIP_CASES = {
    # N = 4096 at eta = 0.70: m = 66, 33 bands (33 strips: one band each)
    "N4096": (dict(N=4096, eta=0.70, delta=0.1, seed=71), (2, 3, 5, 33)),
    # three trials per occupied cell (the run-time trial loop)
    "three_trials": (dict(N=400, eta=0.60, delta=0.2, seed=72, nt=3), (2, 3)),
    # capacity-9 cells (m = 14, seven bands)
    "cap9_cells": (dict(N=300, eta=0.50, delta=0.4, seed=73, cell_min=3.0), (2, 7)),
}


@pytest.mark.parametrize("form", ["fixed", "fp64"])
@pytest.mark.parametrize("case", list(STRIP_CASES))
def test_strip_wavefront(hd, oracle_mod, form, case):
    """Graph wavefront of one replica (hd_opts.strips = K): each strip's
    rebuild and colour passes on its own graph branch, ordered only against
    the two neighbouring strips.  Steps of 7 sweeps (both buffer parities)
    with a measurement each: series, trial counts and every position against
    the oracle, for several K including one band per strip."""
    kw, Ks = STRIP_CASES[case]
    for K in Ks:
        g = hd.HardDisks(kw["N"], kw["eta"], kw["delta"], kw["seed"], precision=form, trials_per_cell=kw.get("nt", 0),
                         cell_min=kw.get("cell_min", 2.0), strips=K)
        o = oracle_mod.OracleChain(kw["N"], kw["eta"], kw["delta"], kw["seed"], form=form, nt=kw.get("nt", 0),
                                   cell_min=kw.get("cell_min", 2.0))
        assert g.geometry()["graph_branches"] == K
        g.run(3, 7, measure=True)
        ser = g.series()
        L = o.geometry()["L"]
        for k in range(3):
            o.sweep(7)
            want = oracle_mod.contact_pressure(o.histogram(50, 1e-3), kw["N"], L, o.realised_dr(1e-3))
            _, rglob = o.psi6()
            assert abs(ser[k, 0, 0] - want["betaP_over_rho"]) <= PRESSURE_TOL * max(1.0, abs(want["betaP_over_rho"]))
            assert complex(ser[k, 0, 2], ser[k, 0, 3]) == rglob
        assert_same_state(g, o)
        g.sweep(3)  # the serial path continues the same chain
        o.sweep(3)
        assert_same_state(g, o)
        g.close()


def test_strip_wavefront_full_size(hd):
    """N = 1024^2 at eta = 0.716 (the benchmark system): the automatic choice
    and an uneven strip count (seven strips of 76 or 77 bands) give the same
    chain as the serial step graph over two steps of 50 sweeps."""
    N = 1024 * 1024
    runs = {}
    for K in (1, 0, 7):
        g = hd.HardDisks(N, 0.716, 0.1, 1, precision="fixed", strips=K)
        gb = g.geometry()["graph_branches"]
        if K == 1:
            assert gb == 1
        elif K == 7:
            assert gb == 7
        else:
            assert gb in (1, 8, 16)  # 16 where the colour pass is 1.5 to 3.5 waves deep (1.85 on GB300), 8 deeper
        g.run(2, 50, measure=True)
        runs[K] = (g.positions(), g.stats(), g.series())
        g.close()
    for K in (0, 7):
        assert np.array_equal(runs[K][0], runs[1][0])
        assert np.array_equal(runs[K][1][0], runs[1][1][0]) and np.array_equal(runs[K][1][1], runs[1][1][1])
        assert np.array_equal(runs[K][2], runs[1][2])


def test_strip_wavefront_shifted_rows_N4194304(hd):
    """N = 2048^2 at eta = 0.720 from the shifted-row lattice with the local
    psi_j field kept per measurement (the fifth configuration's step): the
    automatic strips (8 where the pass is deeper than 3.5 waves) give the
    same chain, series and psi_j field as the serial step graph."""
    import torch
    N = 2048 * 2048
    out = {}
    for K in (1, 0):
        g = hd.HardDisks(N, 0.720, 0.1, 5, precision="fixed", lattice="triangular", strips=K)
        gb = g.geometry()["graph_branches"]
        assert gb == 1 if K == 1 else gb in (1, 8, 16)
        g.run(2, 25, measure=2)
        field = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        g.psi6_local_device(field.data_ptr())
        torch.cuda.synchronize()
        out[K] = (g.positions(), g.series(), g.stats(), field.cpu().numpy())
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2][0], out[1][2][0])
    assert np.array_equal(out[0][3], out[1][3])


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_replica_branches(hd, oracle_mod, form):
    """Replicas of uneven N and eta on concurrent graph branches (the
    default for a batch on the split kernels) against each replica's oracle
    chain, and the same context with the branches off (one batched launch
    per phase) giving the same series and positions."""
    Ns = [16 ** 2, 24 ** 2, 32 ** 2, 20 ** 2, 17 ** 2]
    etas = [0.700, 0.701, 0.702, 0.703, 0.704]
    seeds = [111, 112, 113, 114, 115]
    out = {}
    for rb in (0, 1):
        g = hd.HardDisks(Ns, etas, [0.1] * 5, seeds, precision=form, replica_branches=rb)
        assert g.geometry()["graph_branches"] == (5 if rb == 0 else 1)
        g.run(3, 9, measure=True)
        out[rb] = (g.positions(), g.stats(), g.series())
        g.close()
    os_ = [oracle_mod.OracleChain(n, e, 0.1, sd, form=form) for n, e, sd in zip(Ns, etas, seeds)]
    for o in os_:
        o.sweep(27)
    xy, (att, acc), ser = out[0]
    off = 0
    for r, o in enumerate(os_):
        assert (int(att[r]), int(acc[r])) == o.stats()
        assert np.array_equal(xy[off:off + Ns[r]], o.positions())
        _, rglob = o.psi6()
        assert complex(ser[-1, r, 2], ser[-1, r, 3]) == rglob
        off += Ns[r]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_wavefront_across_draw_tables(hd, oracle_mod, form):
    """Steps of 300 sweeps (two draw tables of 256 and 44 sweeps, each forked
    into branches and joined again) as strips of one replica and as replica
    branches of a batch, against the oracle."""
    g = hd.HardDisks(400, 0.70, 0.1, 81, precision=form, strips=3)
    o = oracle_mod.OracleChain(400, 0.70, 0.1, 81, form=form)
    g.run(1, 300, measure=True)
    o.sweep(300)
    assert_same_state(g, o)
    _, rglob = o.psi6()
    ser = g.series()
    assert complex(ser[0, 0, 2], ser[0, 0, 3]) == rglob
    g.close()
    Ns, etas, seeds = [16 ** 2, 20 ** 2], [0.70, 0.71], [82, 83]
    g = hd.HardDisks(Ns, etas, [0.1] * 2, seeds, precision=form)
    assert g.geometry()["graph_branches"] == 2
    os_ = [oracle_mod.OracleChain(n, e, 0.1, sd, form=form) for n, e, sd in zip(Ns, etas, seeds)]
    g.run(1, 300, measure=False)
    att, acc = g.stats()
    xy = g.positions()
    off = 0
    for r, o in enumerate(os_):
        o.sweep(300)
        assert (int(att[r]), int(acc[r])) == o.stats()
        assert np.array_equal(xy[off:off + Ns[r]], o.positions())
        off += Ns[r]
    g.close()


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_set_positions_full_size(hd, oracle_mod, form):
    """hd_set_positions at N = 1024^2 (cell indices up to 1071): the oracle's
    configuration after two sweeps, a tenth of it moved to periodic images,
    binned on the device equals the oracle's binning, and the chains
    continue together."""
    N = 1024 * 1024
    g, o = make_pair(hd, oracle_mod, form, N, 0.716, 0.1, 3)
    g.sweep(2)  # the sweep counters (keys of the draws) stay; only the positions are replaced
    o.sweep(2)
    xy = o.positions()
    rng = np.random.default_rng(4)
    pick = rng.random(N) < 0.1
    xy[pick] += rng.integers(-3, 4, size=(int(pick.sum()), 2)) * o.geometry()["L"]
    g.set_positions(xy)
    o.set_positions(xy)
    assert np.array_equal(g.positions(), o.positions())
    g.sweep(2)
    o.sweep(2)
    assert np.array_equal(g.positions(), o.positions())


def test_set_positions_with_sigma(hd):
    """With a disk radius sigma != 1, positions are given in length units and
    divided by sigma before binning; in the fixed form every position is a
    multiple of 2^-24 sigma, so handing the positions back is exact."""
    for sigma in (1.5, 0.25):
        g = hd.HardDisks(4096, 0.70, 0.1, 9, sigma=sigma, precision="fixed")
        g.sweep(5)
        xy = g.positions()
        g.set_positions(xy)
        assert np.array_equal(g.positions(), xy)
        g.close()


def test_profiled_steps_of_wavefront_contexts(hd):
    """While profiling, hd_run captures its steps in serial order with a timing
    event around every kernel, also for a context with strips or replica
    branches: the chains stay those of the unprofiled graphs and every
    kernel class of the step is timed."""
    for kw in ({"N": 4096, "eta": 0.70, "delta": 0.1, "seed": 91, "strips": 3},
               {"N": [400, 576], "eta": [0.70, 0.71], "delta": [0.1, 0.1], "seed": [92, 93]}):
        strips = kw.pop("strips", 0)
        a = hd.HardDisks(kw["N"], kw["eta"], kw["delta"], kw["seed"], precision="fixed", strips=strips)
        b = hd.HardDisks(kw["N"], kw["eta"], kw["delta"], kw["seed"], precision="fixed", strips=strips)
        assert a.geometry()["graph_branches"] > 1
        a.profile(True)
        a.run(2, 7, measure=True)
        kt = a.kernel_times()
        a.profile(False)
        b.run(2, 7, measure=True)
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.series(), b.series())
        for cls in ("rebuild", "pass", "hist", "psi6"):
            assert kt[cls][0] > 0.0 and kt[cls][1] > 0
        assert kt["pass"][1] == 2 * 7 * 4  # whole passes: the profiled graph has no strips
        a.close()
        b.close()
