"""Pins of the oracle's contact-shell pair histogram (Eq. 2 numerator)
against brute-force enumeration from global coordinates."""
import numpy as np
import pytest

from helpers import FX, min_image_d2, min_image_d2_fixed, to_fixed


@pytest.mark.parametrize("K,dr", [(50, 1e-3), (100, 1e-3), (40, 0.01)])
def test_fixed_histogram_exact_from_global(oracle_mod, K, dr):
    o = oracle_mod.OracleChain(400, 0.70, 0.12, 3, form="fixed")
    o.sweep(40)
    g = o.geometry()
    h = o.histogram(K, dr)
    assert np.array_equal(h, o.histogram(K, dr, brute=True))
    r2 = min_image_d2_fixed(to_fixed(o.positions()), g["LF"])
    iu = np.triu_indices(400, 1)
    r2 = r2[iu]
    DR = int(round(dr * FX))
    edges = np.array([((1 << 25) + k * DR) ** 2 for k in range(K + 1)], dtype=np.int64)
    want = np.histogram(r2, bins=edges)[0]
    # numpy's last bin is closed; the oracle's is half-open
    want[-1] -= np.count_nonzero(r2 == edges[-1])
    assert np.array_equal(h, want.astype(np.uint64))
    assert h.sum() > 0


def test_fp64_histogram_matches_global(oracle_mod):
    o = oracle_mod.OracleChain(400, 0.70, 0.12, 4, form="fp64")
    o.sweep(40)
    g = o.geometry()
    K, dr = 100, 1e-3
    h = o.histogram(K, dr)
    assert np.array_equal(h, o.histogram(K, dr, brute=True))
    r = np.sqrt(min_image_d2(o.positions(), g["L"])[np.triu_indices(400, 1)])
    want = np.histogram(r, bins=2.0 + dr * np.arange(K + 1))[0]
    # frame arithmetic differs from global arithmetic only at the last ulp
    assert np.abs(h.astype(np.int64) - want).sum() <= 2
