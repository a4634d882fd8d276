"""The 1024-word-row latency split (row_ops 4): bit-exact against the CPU
oracle at every size it serves (N = 2^10 .. 2^17: one row kernel at 2^10,
one cluster launch per batch at 2^11 .. 2^13, three launches from 2^14),
both word types, Eq. 2 and Algorithm 8, both scaling modes, plus aliasing,
edge inputs, moduli near the word limits, larger batches, CUDA graph
capture and the allocation-free entry point."""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, schoolbook_coeff, to_dev, to_host

pytestmark = pytest.mark.gpu

WIDE_POLYMUL = [10, 11, 12, 13, 14, 15, 16, 17]


def _plan(log2n, nlimbs, qbits=60, halving=False, fused=False):
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(log2n, nlimbs, qbits)
    plan = Plan(1 << log2n, qs, psis, halving=halving, fused=fused)
    capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT, row_ops=4)
    return plan, qs, psis


@pytest.mark.parametrize("fused", [False, True], ids=["eq2", "alg8"])
@pytest.mark.parametrize("halving", [False, True], ids=["fold", "halving"])
@pytest.mark.parametrize("log2n", WIDE_POLYMUL)
def test_wide_polymul_batches(oracle, log2n, halving, fused):
    """Several polynomials and limbs in one launch: every unit in full."""
    n = 1 << log2n
    L, P = (4, 3) if log2n <= 15 else (3, 2)
    plan, qs, psis = _plan(log2n, L, halving=halving, fused=fused)
    a, b = operands(70000 + log2n, qs, P, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got, oracle_polymul_batch(oracle, a, b, qs, psis))


@pytest.mark.parametrize("fused", [False, True], ids=["eq2", "alg8"])
@pytest.mark.parametrize("log2n", WIDE_POLYMUL)
def test_wide_aliasing(oracle, log2n, fused):
    """c may alias a or b; a == b (squaring, one column transform)."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2, fused=fused)
    a, b = operands(71000 + log2n, qs, 1, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    want_sq = oracle_polymul_batch(oracle, a, a, qs, psis)
    da, db = to_dev(a), to_dev(b)
    plan.polymul(da, db, out=da)
    assert np.array_equal(to_host(da), want)
    da, db = to_dev(a), to_dev(b)
    plan.polymul(da, db, out=db)
    assert np.array_equal(to_host(db), want)
    da = to_dev(a)
    assert np.array_equal(to_host(plan.polymul(da, da)), want_sq)
    plan.polymul(da, da, out=da)
    assert np.array_equal(to_host(da), want_sq)


@pytest.mark.parametrize("log2n", WIDE_POLYMUL)
def test_wide_edges(oracle, log2n):
    """Zeros, maximal words (all q - 1), monomials across the X^N = -1 wrap,
    sampled schoolbook coefficients."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 1)
    q = qs[0]
    z = np.zeros((1, 1, n), np.uint64)
    full = np.full((1, 1, n), q - 1, np.uint64)
    assert not to_host(plan.polymul(to_dev(z), to_dev(full))).any()
    got = to_host(plan.polymul(to_dev(full), to_dev(full)))
    assert np.array_equal(got[0, 0], np.array([(2 * k + 2 - n) % q for k in range(n)], np.uint64))
    rng = np.random.default_rng(log2n)
    for i, j in [(0, 0), (n - 1, n - 1), (n - 1, 1), (1023, 1), tuple(rng.integers(0, n, 2))]:
        a = np.zeros((1, 1, n), np.uint64)
        b = np.zeros((1, 1, n), np.uint64)
        a[0, 0, i] = 1
        b[0, 0, j] = 1
        want = np.zeros(n, np.uint64)
        if i + j < n:
            want[i + j] = 1
        else:
            want[i + j - n] = q - 1
        assert np.array_equal(to_host(plan.polymul(to_dev(a), to_dev(b)))[0, 0], want), (i, j)
    a, b = operands(72000 + log2n, qs, 1, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    for k in rng.integers(0, n, 3):
        assert int(got[0, 0, k]) == schoolbook_coeff(a[0, 0], b[0, 0], q, int(k))


@pytest.mark.parametrize("qbits,log2n", [(62, 10), (62, 12), (62, 16), (30, 13), (30, 14), (40, 17)])
def test_wide_word_sizes(oracle, qbits, log2n):
    """Moduli at the top of the 64-bit range (lazy words up to 4q < 2^64)
    and small ones in 64-bit words."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2, qbits=qbits)
    a, b = operands(73000 + log2n + qbits, qs, 1, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got, oracle_polymul_batch(oracle, a, b, qs, psis))
    d = to_dev(a)
    plan.ntt_fwd_(d)
    fwd = to_host(d)
    for l in range(2):
        assert np.array_equal(fwd[0, l], oracle.ntt_fwd_bo(a[0, l], qs[l], psis[l])), l
    plan.ntt_inv_(d)
    assert np.array_equal(to_host(d), a)


@pytest.mark.parametrize("log2n", [10, 12, 14, 17])
def test_wide_graph(oracle, log2n):
    """A polymul captured with the wide tuning replays bit-exactly after the
    inputs change."""
    plan, qs, psis = _plan(log2n, 2)
    a, b = operands(74000 + log2n, qs, 2, 1 << log2n)
    da, db = to_dev(a), to_dev(b)
    dc = da.new_empty(da.shape)
    g = plan.graph_polymul(da, db, dc)
    for rep in range(2):
        if rep:
            a, b = operands(74100 + log2n, qs, 2, 1 << log2n)
            da.copy_(to_dev(a))
            db.copy_(to_dev(b))
        g.launch()
        plan.sync()
        assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis)), rep
    g.close()


@pytest.mark.parametrize("log2n", [10, 13, 14, 16])
def test_wide_noalloc(oracle, log2n):
    import torch
    from paper_2209_01290_gb300 import capi
    plan, qs, psis = _plan(log2n, 2)
    a, b = operands(75000 + log2n, qs, 2, 1 << log2n)
    da, db = to_dev(a), to_dev(b)
    dc = torch.empty_like(da)
    capi.pm_polymul_noalloc(plan.handle, da.data_ptr(), db.data_ptr(), dc.data_ptr(), 2,
                            torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis))


def test_wide_phase_events():
    """The profiling hook records one event per launch of the split."""
    import torch
    from paper_2209_01290_gb300 import capi
    plan, qs, psis = _plan(16, 1)
    a, b = operands(76000, qs, 1, 1 << 16)
    da, db = to_dev(a), to_dev(b)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev:
        e.record()  # torch creates the CUDA event at its first record
    torch.cuda.synchronize()
    capi.pm_plan_set_phase_events(plan.handle, [e.cuda_event for e in ev])
    plan.polymul(da, db)
    capi.pm_plan_set_phase_events(plan.handle, [])
    torch.cuda.synchronize()
    assert all(ev[k].elapsed_time(ev[k + 1]) >= 0 for k in range(3))


def test_wide_tuning_range():
    from paper_2209_01290_gb300 import capi
    plan, *_ = _plan(14, 1)
    assert capi.pm_plan_get_tuning(plan.handle).row_ops == 4
    with pytest.raises(capi.PMError) as e:
        capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT, row_ops=6)
    assert e.value.status == -1


def test_resolved_row_kernel_rule():
    """pm_plan_resolve_tuning reports the rule pm.h states for row_ops 0:
    1024-word rows for 64-bit words except N = 2^12 above 64 units (then
    1024-thread rows up to one row per SM, two-operand rows above); 32-bit
    words: 1024-word rows up to 2^20 words per batch.  A set row_ops is kept."""
    import torch
    from paper_2209_01290_gb300 import Plan, capi
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cases = [(12, 1, False), (12, 64, False), (12, 65, False), (12, sms, False),
             (12, sms + 1, False), (16, 1, False), (16, 4096, False), (10, 4096, False),
             (16, 16, True), (16, 17, True), (12, 256, True), (12, 257, True)]
    for log2n, npoly, w32 in cases:
        qs, psis = capi.pm_find_params(log2n, 1, 30 if w32 else 60)
        plan = Plan(1 << log2n, qs, psis, word32=w32)
        got = capi.pm_plan_resolve_tuning(plan.handle, npoly).row_ops
        if (npoly << log2n) <= (1 << 20) if w32 else not (log2n == 12 and npoly > 64):
            want = 4
        else:
            want = 3 if (npoly << max(log2n - 12, 0)) <= sms else 2
        assert got == want, (log2n, npoly, w32, got)
        assert capi.pm_plan_get_tuning(plan.handle).row_ops == 0
        capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT, row_ops=1)
        assert capi.pm_plan_resolve_tuning(plan.handle, npoly).row_ops == 1
    with pytest.raises(capi.PMError):
        capi.pm_plan_resolve_tuning(plan.handle, 0)


def test_short_twiddles_times_out_then_recovers(oracle):
    """Host-side fault injection on the bulk-copy wait of the row kernel:
    every row CTA's barrier expects 16 bytes more than its twiddle copies
    deliver, so each bounded wait gives up after about a second and the CTA
    skips its row; pm_plan_sync reports PM_ERR_TIMEOUT.  The next call is
    correct and reports no error."""
    import time
    from paper_2209_01290_gb300 import capi
    plan, qs, psis = _plan(16, 1)
    a, b = operands(77000, qs, 1, 1 << 16)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    da, db = to_dev(a), to_dev(b)
    capi.pm_plan_inject_fault(plan.handle, capi.PM_FAULT_SHORT_TWIDDLES)
    t0 = time.time()
    plan.polymul(da, db)
    with pytest.raises(capi.PMError) as e:
        plan.sync()
    assert e.value.status == -7
    assert time.time() - t0 < 30
    got = to_host(plan.polymul(da, db))
    plan.sync()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("fused", [False, True], ids=["eq2", "alg8"])
@pytest.mark.parametrize("qbits", [60, 62])
@pytest.mark.parametrize("log2n", [14, 15, 16, 17])
def test_wide_tensor_copy_columns(oracle, log2n, qbits, fused):
    """row_ops 5: the column kernels load their tiles with 2-D tensor copies
    (and the inverse one stores with one).  Products (distinct operands,
    aliased output, squares), forward and inverse NTTs: every word against
    the oracle.  62-bit primes take the classic lazy ranges, 60-bit the
    wide ones.  32 units avoid the one-launch cluster path at N = 2^14."""
    from paper_2209_01290_gb300 import Plan, capi
    import oracle as orc
    n = 1 << log2n
    L, P = (2, 16) if log2n <= 15 else (2, 2)
    qs, psis = capi.pm_find_params(log2n, L, qbits)
    plan = Plan(n, qs, psis, fused=fused)
    capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT, row_ops=5)
    a, b = operands(78000 + log2n + qbits, qs, P, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    da, db = to_dev(a), to_dev(b)
    assert np.array_equal(to_host(plan.polymul(da, db)), want)
    plan.polymul(da, db, out=db)
    assert np.array_equal(to_host(db), want)
    da = to_dev(a)
    assert np.array_equal(to_host(plan.polymul(da, da)),
                          oracle_polymul_batch(oracle, a, a, qs, psis))
    x = to_dev(a[:1])
    plan.ntt_fwd_(x)
    for l in range(L):
        assert np.array_equal(to_host(x)[0, l], orc.ntt_fwd_bo(a[0, l], qs[l], psis[l]))
    plan.ntt_inv_(x)
    assert np.array_equal(to_host(x), a[:1])
    plan.sync()
