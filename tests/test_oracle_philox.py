"""Pin the oracle's Philox4x32-10 to the published known-answer vectors."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle_mod.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_counter_sensitivity(oracle_mod):
    # a bijection of the counter for a fixed key: distinct counters, distinct blocks
    outs = {tuple(oracle_mod.philox4x32_10([i, 0, 0, 0], [1, 2]).tolist()) for i in range(256)}
    assert len(outs) == 256
    # uniformity sanity of the words (mean of U(0,1) over 4096 words)
    w = np.concatenate([oracle_mod.philox4x32_10([i, 7, 9, 3], [5, 6]) for i in range(1024)])
    assert abs(w.astype(np.float64).mean() / 2**32 - 0.5) < 0.02
