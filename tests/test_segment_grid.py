"""Host check of the segment grid that the bulk-copy pass and the persistent
sweep decode on the device (hd_api.cu plans it, hd_pass_tma.cu and
hd_persist.cu decode it): for the geometries of the tests, the benchmark and
the equation-of-state scan, and every block size, every item's band,
half-column range and derived cell indices lie inside the replica's planes,
every active cell is covered exactly once per phase, and the progress word of
every band exists.  The planning arithmetic is restated here from the
library's definitions: m = the largest even integer with L/m >= the minimum
cell side, hm = m / 2, nseg = ceil(hm / threads), segw = ceil(hm / nseg).  The device divides by nseg (and by hm, and by the
tile count per row) with a multiply-high by an invariant reciprocal
(Granlund and Montgomery, "Division by invariant integers using
multiplication", 1994, Sec. 4): q = (t + ((n - t) >> 1)) >> (l - 1) with
t = mulhi(mul, n), l = ceil(log2 d) and mul = floor(2^32 (2^l - d) / d) + 1;
that decode is checked against integer division here too."""
import math

import numpy as np
import pytest


def magic(d):
    l = 0
    while (1 << l) < d:
        l += 1
    return ((((1 << l) - d) << 32) // d + 1) & 0xFFFFFFFF, l - 1


def div_by(n, mul, sh):
    t = (mul * n) >> 32
    return (t + ((n - t) >> 1)) >> sh


def cells_per_side(N, eta, cell_min=2.0):
    L = math.sqrt(N * math.pi / eta)
    return 2 * int(L / (2 * cell_min))


def plan(ms, threads):
    reps, blk_seg, band0 = [], 0, 0
    for m in ms:
        hm = m // 2
        nseg = (hm + threads - 1) // threads
        segw = (hm + nseg - 1) // nseg
        reps.append(dict(m=m, hm=hm, hh=hm * hm, nseg=nseg, segw=segw, blk_seg=blk_seg, band0=band0))
        blk_seg += hm * nseg
        band0 += hm
    return reps, blk_seg, band0


GEOMETRIES = {
    "config1": [cells_per_side(256, 0.70)],
    "ragged_N1000": [cells_per_side(1000, 0.55)],
    "two_disks": [cells_per_side(2, 2 * math.pi / 100)],
    "cap9": [cells_per_side(300, 0.50, 3.0)],
    "config2": [cells_per_side(65536, 0.708)],
    "config3": [cells_per_side(1 << 20, 0.716)],
    "config5": [cells_per_side(1 << 22, 0.720)],
    "N4096sq": [cells_per_side(1 << 24, 0.716)],
    "replicas5": [cells_per_side(n, e) for n, e in zip([256, 576, 1024, 400, 289],
                                                        [0.700, 0.701, 0.702, 0.703, 0.704])],
    "scan31": [cells_per_side([128 ** 2, 192 ** 2, 256 ** 2, 384 ** 2, 512 ** 2][r % 5], 0.700 + 0.001 * r)
               for r in range(31)],
}


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
@pytest.mark.parametrize("name", list(GEOMETRIES))
def test_segment_items_cover_every_active_cell_once(name, threads):
    ms = GEOMETRIES[name]
    assert all(m >= 4 and m % 2 == 0 for m in ms)
    reps, NI, bands = plan(ms, threads)
    seen = [set() for _ in reps]
    for idx in range(NI):
        r = max(i for i, rep in enumerate(reps) if rep["blk_seg"] <= idx)
        rep = reps[r]
        loc = idx - rep["blk_seg"]
        b = div_by(loc, *magic(rep["nseg"])) if rep["nseg"] > 1 else loc
        assert b == loc // rep["nseg"]
        X0 = (loc - b * rep["nseg"]) * rep["segw"]
        Bv = min(rep["segw"], rep["hm"] - X0)
        assert 0 <= b < rep["hm"] and Bv >= 1 and X0 + Bv <= rep["hm"]
        assert rep["segw"] <= threads  # one half-column per thread
        assert 2 + rep["band0"] + b < 2 + bands
        for x in range(X0, X0 + Bv):
            a = b * rep["hm"] + x
            assert a < rep["hh"]
            assert 3 * rep["hh"] + a < rep["m"] ** 2  # the rebuild's fourth plane
            assert (b, x) not in seen[r]
            seen[r].add((b, x))
    for r, rep in enumerate(reps):
        assert len(seen[r]) == rep["hh"]


def test_invariant_divisor_decode_matches_integer_division():
    rng = np.random.default_rng(7)
    ns = np.concatenate([np.arange(0, 4096), rng.integers(0, 1 << 31, 4096),
                         np.array([(1 << 31) - 1, (1 << 32) - 1])]).astype(np.uint64)
    for d in list(range(2, 1100)) + [2047, 2048, 2049, 4095, 4096, 65535, 65536, 1 << 20, (1 << 31) - 1]:
        mul, sh = magic(d)
        t = (np.uint64(mul) * ns) >> np.uint64(32)
        q = (t + ((ns - t) >> np.uint64(1))) >> np.uint64(sh)
        assert np.array_equal(q, ns // np.uint64(d)), d
