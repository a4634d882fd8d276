"""Fused polynomial multiplication (Algorithm 8, plan flag PM_PLAN_FUSED):
bit-exact against the oracle on every code path, both scaling modes and
both launch variants, plus the edge cases of the pair step (the sign
(-1)^i, maximal words, N = 4) and the uneven, graph and serving paths."""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, schoolbook_coeff, to_dev, to_host

pytestmark = pytest.mark.gpu

FUSED_LOG2N = list(range(2, 18))


def _plan(log2n, nlimbs, qbits=60, halving=False, variant=None):
    """variant: None (the plan's default launch) or (variant, row_ops)."""
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(log2n, nlimbs, qbits)
    plan = Plan(1 << log2n, qs, psis, halving=halving, fused=True)
    if variant is not None:
        capi.pm_plan_tune(plan.handle, variant[0], row_ops=variant[1])
    return plan, qs, psis


@pytest.mark.parametrize("variant", [(0, 1), (0, 2), (0, 3), (0, 4), (1, 1)],
                         ids=["split-rows1", "split-rows2", "split-rowslat", "split-wide",
                              "persistent"])
@pytest.mark.parametrize("halving", [False, True], ids=["fold2N", "halving"])
@pytest.mark.parametrize("log2n", FUSED_LOG2N)
def test_fused_all_sizes(oracle, log2n, halving, variant):
    """N = 4 .. 2^17 through k_small, k_rows (2^12), k_fused13 and the column
    split (three launches or one persistent launch); 2 polys x 3 limbs."""
    n = 1 << log2n
    L, P = (3, 2) if log2n <= 15 else (2, 1)
    plan, qs, psis = _plan(log2n, L, halving=halving, variant=variant)
    a, b = operands(41000 + log2n, qs, P, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("log2n", [4, 12, 16])
def test_fused_matches_alg8_oracle(oracle, log2n):
    """The oracle's own Algorithm 8 gives the same words."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 1)
    a, b = operands(42000 + log2n, qs, 1, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got[0, 0], oracle.polymul_alg8(a[0, 0], b[0, 0], qs[0], psis[0]))


@pytest.mark.parametrize("halving", [False, True], ids=["fold2N", "halving"])
@pytest.mark.parametrize("log2n", [12, 14, 16, 17])
def test_fused_rows_one_after_other(oracle, log2n, halving):
    """Row kernel with the operands transformed one after the other
    (row_ops = 1), one limb pair per product."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2, halving=halving, variant=(0, 1))
    a, b = operands(43000 + log2n, qs, 1, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got, oracle_polymul_batch(oracle, a, b, qs, psis))


@pytest.mark.parametrize("log2n", [2, 3, 11, 12, 13, 16])
def test_fused_edges(oracle, log2n):
    """Maximal words (q-1 everywhere), monomials whose product wraps with a
    sign, and single nonzero pairs at odd and even pair indices (both signs
    of the pair step)."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 1)
    q = qs[0]
    full = np.full((1, 1, n), q - 1, np.uint64)
    got = to_host(plan.polymul(to_dev(full), to_dev(full)))
    want = np.array([(2 * k + 2 - n) % q for k in range(n)], dtype=np.uint64)
    assert np.array_equal(got[0, 0], want)
    rng = np.random.default_rng(log2n)
    for i, j in [(0, 0), (n - 1, n - 1), (n - 1, 1), (1, n - 2), tuple(rng.integers(0, n, 2))]:
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
    a, b = operands(44000 + log2n, qs, 1, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    for k in rng.integers(0, n, 4):
        assert int(got[0, 0, k]) == schoolbook_coeff(a[0, 0], b[0, 0], q, int(k))


@pytest.mark.parametrize("qbits,log2n", [(62, 12), (62, 16), (30, 13), (30, 16)])
def test_fused_word_sizes(oracle, qbits, log2n):
    """62-bit moduli (sums a0 + a1 near 2^63) and 30-bit moduli."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2, qbits)
    a, b = operands(45000 + qbits + log2n, qs, 1, n)
    assert np.array_equal(to_host(plan.polymul(to_dev(a), to_dev(b))),
                          oracle_polymul_batch(oracle, a, b, qs, psis))


@pytest.mark.parametrize("log2n", [12, 13, 16])
def test_fused_aliasing(oracle, log2n):
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2)
    a, b = operands(46000 + log2n, qs, 1, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    want_sq = oracle_polymul_batch(oracle, a, a, qs, psis)
    da, db = to_dev(a), to_dev(b)
    plan.polymul(da, db, out=db)
    assert np.array_equal(to_host(db), want)
    da = to_dev(a)
    plan.polymul(da, da, out=da)
    assert np.array_equal(to_host(da), want_sq)


def test_fused_ntt_unchanged(oracle):
    """The flag changes products only: pm_ntt_fwd / pm_ntt_inv stay the
    full transforms (1/N, not 2/N)."""
    log2n = 14
    plan, qs, psis = _plan(log2n, 1)
    x, _ = operands(47000, qs, 1, 1 << log2n)
    d = to_dev(x)
    plan.ntt_fwd_(d)
    assert np.array_equal(to_host(d)[0, 0], oracle.ntt_fwd_bo(x[0, 0], qs[0], psis[0]))
    plan.ntt_inv_(d)
    assert np.array_equal(to_host(d), x)


def test_fused_flag_checks():
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(1, 1, 60)
    with pytest.raises(capi.PMError) as ei:
        Plan(2, qs, psis, fused=True)
    assert capi.STATUS_NAMES[ei.value.status] == "PM_ERR_N"
    plan, _, _ = _plan(5, 1, halving=True)
    assert capi.pm_plan_flags(plan.handle) == capi.PM_PLAN_FUSED | capi.PM_PLAN_HALVING


def test_fused_graph(oracle):
    import torch
    plan, qs, psis = _plan(16, 2)
    a, b = operands(48000, qs, 2, 1 << 16)
    da, db = to_dev(a), to_dev(b)
    dc = torch.empty_like(da)
    g = plan.graph_polymul(da, db, dc)
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis))


@pytest.mark.parametrize("mode", [1, 2], ids=["persistent", "grouped"])
def test_fused_uneven(oracle, mode):
    """An uneven batch of fused plans; mixing fused and default plans of
    N >= 4096 in one launch is rejected."""
    from paper_2209_01290_gb300 import Plan, Queue, capi
    shapes = [(12, 2), (16, 1), (13, 3), (5, 2), (14, 2), (17, 1)]
    q = Queue(mode=mode)
    jobs, data = [], []
    for j, (log2n, L) in enumerate(shapes):
        plan, qs, psis = _plan(log2n, L)
        a, b = operands(49000 + j, qs, 1, 1 << log2n)
        da, db = to_dev(a), to_dev(b)
        dc = da.new_empty(da.shape)
        jobs.append((plan, da, db, dc))
        data.append((a, b, qs, psis, dc))
    q.polymul_uneven(jobs)
    q.sync()
    for a, b, qs, psis, dc in data:
        assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis))
    qs, psis = capi.pm_find_params(14, 1, 60)
    plain = Plan(1 << 14, qs, psis)
    a, b = operands(49100, qs, 1, 1 << 14)
    da, db = to_dev(a), to_dev(b)
    with pytest.raises(capi.PMError):
        q.polymul_uneven(jobs[:2] + [(plain, da, db, da.new_empty(da.shape))])


def test_fused_server_mixed_kinds(oracle):
    """Requests on fused, halving and default plans interleaved: the server
    splits batches by plan kind and every result equals the product."""
    import torch
    from paper_2209_01290_gb300 import Plan, capi
    from test_gpu_serving import _copy_out
    kinds = [dict(), dict(fused=True), dict(halving=True), dict(fused=True, halving=True)]
    plans = []
    for k, kw in enumerate(kinds):
        for log2n, L in [(13, 2), (16, 1)]:
            qs, psis = capi.pm_find_params(log2n, L, 60)
            plans.append((Plan(1 << log2n, qs, psis, **kw), qs, psis))
    reqs = []
    for i in range(24):
        plan, qs, psis = plans[i % len(plans)]
        a, b = operands(49500 + i, qs, 1, plan.n)
        reqs.append((plan, to_dev(a), to_dev(b), oracle_polymul_batch(oracle, a, b, qs, psis)))
    torch.cuda.synchronize()
    srv = capi.pm_server_create(0, 512 << 20, 0, 2)
    ids = [capi.pm_server_submit(srv, p.handle, da.data_ptr(), db.data_ptr(), 1)
           for p, da, db, _ in reqs]
    for i, (plan, da, db, want) in enumerate(reqs):
        ptr, _ = capi.pm_server_wait(srv, ids[i])
        assert np.array_equal(to_host(_copy_out(ptr, da.shape)), want), i
        capi.pm_server_release(srv, ids[i])
    capi.pm_server_destroy(srv)
