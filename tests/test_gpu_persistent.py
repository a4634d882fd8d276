"""The persistent work-queue polymul: many units, pipeline lags, tuning
checks, and the bounded-wait error path (a dependency signal withheld on the
host side; the waits run out, the host reads PM_ERR_TIMEOUT, later calls
work)."""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, to_dev, to_host

pytestmark = pytest.mark.gpu


def _setup(log2n, L, P, seed):
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(log2n, L, 60)
    plan = Plan(1 << log2n, qs, psis)
    a, b = operands(seed, qs, P, 1 << log2n)
    return plan, qs, psis, a, b


@pytest.mark.parametrize("log2n,L,P", [(13, 4, 16), (14, 3, 8), (15, 2, 8), (16, 4, 6), (17, 2, 3)])
@pytest.mark.parametrize("lags", [(1, 2), (8, 16), (40, 90)])
@pytest.mark.parametrize("row_ops", [0, 1], ids=["rows1024", "rows4096"])
def test_persistent_lags(oracle, log2n, L, P, lags, row_ops):
    """Results do not depend on the pipeline distances, on the CTA count or
    on the task size (1024-word split, the default, or 4096-word rows);
    every unit is checked against the oracle (units > lag exercise the
    steady state, units < lag the prologue/epilogue)."""
    from paper_2209_01290_gb300 import capi
    plan, qs, psis, a, b = _setup(log2n, L, P, 11000 + log2n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    for ctas in (1, 4):
        capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_PERSISTENT, ctas, lags[0], lags[1],
                          row_ops=row_ops)
        got = to_host(plan.polymul(to_dev(a), to_dev(b)))
        plan.sync()
        assert np.array_equal(got, want), (ctas, lags)


def test_tuning_validation():
    from paper_2209_01290_gb300 import capi
    plan, *_ = _setup(14, 1, 1, 1)
    t = capi.pm_plan_get_tuning(plan.handle)
    assert t.variant == capi.PM_VARIANT_SPLIT and t.ctas_per_sm == 3 and t.row_ops == 0
    for bad in [(capi.PM_VARIANT_PERSISTENT, 0, 8, 16), (capi.PM_VARIANT_PERSISTENT, 3, 8, 8),
                (capi.PM_VARIANT_PERSISTENT, 5, 8, 16), (7, 3, 8, 16)]:
        with pytest.raises(capi.PMError) as e:
            capi.pm_plan_tune(plan.handle, *bad)
        assert e.value.status == -1
    capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT)
    assert capi.pm_plan_get_tuning(plan.handle).variant == capi.PM_VARIANT_SPLIT


def test_withheld_signal_times_out_then_recovers(oracle):
    """Host-side fault injection: the row tasks of the next launch wait for a
    signal that never comes.  Each wait gives up after about a second, the
    launch ends, pm_plan_sync reports PM_ERR_TIMEOUT; the next call is
    correct and reports no error."""
    import time
    from paper_2209_01290_gb300 import capi
    plan, qs, psis, a, b = _setup(14, 1, 2, 12000)
    capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_PERSISTENT)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    da, db = to_dev(a), to_dev(b)
    capi.pm_plan_inject_fault(plan.handle, capi.PM_FAULT_WITHHOLD_SIGNAL)
    t0 = time.time()
    plan.polymul(da, db)
    with pytest.raises(capi.PMError) as e:
        plan.sync()
    assert e.value.status == -7
    assert time.time() - t0 < 30
    got = to_host(plan.polymul(da, db))
    plan.sync()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", [0, 1], ids=["split", "persistent"])
@pytest.mark.parametrize("log2n", [12, 13, 16, 17])
def test_graph_replay(oracle, log2n, variant):
    """A captured polymul replays bit-exactly, also after the inputs change."""
    from paper_2209_01290_gb300 import capi
    plan, qs, psis, a, b = _setup(log2n, 2, 2, 13000 + log2n)
    capi.pm_plan_tune(plan.handle, variant)
    da, db = to_dev(a), to_dev(b)
    dc = da.new_empty(da.shape)
    g = plan.graph_polymul(da, db, dc)
    for rep in range(2):
        if rep:
            a, b = operands(13100 + log2n, qs, 2, 1 << log2n)
            da.copy_(to_dev(a))
            db.copy_(to_dev(b))
        g.launch()
        plan.sync()
        assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis)), rep
    g.close()


@pytest.mark.parametrize("log2n,L,P", [(12, 2, 4), (14, 2, 8), (16, 4, 8)])
def test_autotune_picks_a_valid_choice(oracle, log2n, L, P):
    from paper_2209_01290_gb300 import capi
    plan, qs, psis, a, b = _setup(log2n, L, P, 14000 + log2n)
    t, ms = capi.pm_plan_autotune(plan.handle, P)
    assert ms > 0 and t.variant in (0, 1)
    got = capi.pm_plan_get_tuning(plan.handle)
    assert (got.variant, got.row_ops, got.lag_fwd) == (t.variant, t.row_ops, t.lag_fwd)
    out = to_host(plan.polymul(to_dev(a), to_dev(b)))
    plan.sync()
    assert np.array_equal(out, oracle_polymul_batch(oracle, a, b, qs, psis))
