"""Error paths of the device kernels, exercised without faulting anything.

The bulk-copy colour pass checks its staging plan (16-byte aligned starts and
slot planes, sizes within its shared-memory areas) before it issues a copy.
The environment variable HD_TEST_UNALIGNED_SLOT_STRIDE=1 makes a context
whose slot planes are 8 cells further apart than the 16-cell boundary the
plan needs: every block then rejects its plan, issues no copy, skips its
cells and raises the error flag, which the host reports as HD_ERR_TIMEOUT
and keeps sticky.  The same layout is valid for the cp.async pass, which is
checked against the oracle to show that only the staging plan is refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import paper_1211_1645_gb300 as hd
    hd.load()
    return hd


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_refused_staging_plan_reports_timeout_and_sticks(hd, monkeypatch, form):
    from paper_1211_1645_gb300.hd import HD_ERR_STATE, HD_ERR_TIMEOUT, HDError
    monkeypatch.setenv("HD_TEST_UNALIGNED_SLOT_STRIDE", "1")
    g = hd.HardDisks(1000, 0.70, 0.1, 3, precision=form, sweep_kernel="tma")
    monkeypatch.delenv("HD_TEST_UNALIGNED_SLOT_STRIDE")
    before = g.positions()
    g.sweep(1)
    with pytest.raises(HDError) as e:
        g.stats()
    assert e.value.status == HD_ERR_TIMEOUT
    for call in (lambda: g.sweep(1), g.positions, g.stats):
        with pytest.raises(HDError) as e:
            call()
        assert e.value.status == HD_ERR_STATE
    g.close()
    # a fresh context without the hook runs the same chain normally
    g2 = hd.HardDisks(1000, 0.70, 0.1, 3, precision=form, sweep_kernel="tma")
    assert np.array_equal(g2.positions(), before)
    g2.sweep(2)
    assert int(g2.stats()[0][0]) > 0
    g2.close()


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_unaligned_slot_stride_is_valid_for_the_cp_async_pass(hd, oracle_mod, monkeypatch, form):
    monkeypatch.setenv("HD_TEST_UNALIGNED_SLOT_STRIDE", "1")
    g = hd.HardDisks(1000, 0.70, 0.1, 3, precision=form, sweep_kernel="split")
    monkeypatch.delenv("HD_TEST_UNALIGNED_SLOT_STRIDE")
    o = oracle_mod.OracleChain(1000, 0.70, 0.1, 3, form=form)
    g.sweep(25)
    o.sweep(25)
    att, acc = g.stats()
    assert (int(att[0]), int(acc[0])) == o.stats()
    assert np.array_equal(g.positions(), o.positions())
    g.close()


@pytest.mark.parametrize("form", ["fixed", "fp64"])
def test_persistent_sweep_wait_gives_up_and_sticks(hd, monkeypatch, form):
    """HD_TEST_PERSIST_STALL=1 at creation: the persistent sweep never
    publishes the first item of band 0, and its bounded dependency waits give
    up after 4096 polls instead of waiting forever.  The launch ends, the
    host reports HD_ERR_TIMEOUT and the context stays in its error state."""
    from paper_1211_1645_gb300.hd import HD_ERR_STATE, HD_ERR_TIMEOUT, HDError
    monkeypatch.setenv("HD_TEST_PERSIST_STALL", "1")
    g = hd.HardDisks(4096, 0.70, 0.1, 3, precision=form, sweep_kernel="persistent")
    monkeypatch.delenv("HD_TEST_PERSIST_STALL")
    g.sweep(3)
    with pytest.raises(HDError) as e:
        g.stats()
    assert e.value.status == HD_ERR_TIMEOUT
    with pytest.raises(HDError) as e:
        g.sweep(1)
    assert e.value.status == HD_ERR_STATE
    g.close()
    g2 = hd.HardDisks(4096, 0.70, 0.1, 3, precision=form, sweep_kernel="persistent")
    g2.sweep(3)
    assert int(g2.stats()[0][0]) > 0
    g2.close()
