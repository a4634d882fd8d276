"""32-bit-word path (PM_PLAN_WORD32, q < 2^30): bit-exact against the CPU
oracle (which works on the same values in 64-bit words) on every code path,
both scaling modes, Eq. 2 and Algorithm 8, both row kernels, plus the edge
cases and the word-size checks of the C ABI."""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, schoolbook_coeff

pytestmark = pytest.mark.gpu

ALL_LOG2N = list(range(1, 18))


def to_dev32(x: np.ndarray):
    import torch
    x32 = np.ascontiguousarray(x.astype(np.uint32))
    return torch.from_numpy(x32.view(np.int32)).to("cuda:0")


def to_host32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32).astype(np.uint64)


def _plan(log2n, nlimbs, qbits=30, halving=False, fused=False, row_ops=None):
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(log2n, nlimbs, qbits)
    plan = Plan(1 << log2n, qs, psis, halving=halving, fused=fused, word32=True)
    if row_ops is not None:
        capi.pm_plan_tune(plan.handle, capi.PM_VARIANT_SPLIT, row_ops=row_ops)
    return plan, qs, psis


@pytest.mark.parametrize("row_ops", [1, 2, 3, 4], ids=["rows1", "rows2", "rowslat", "wide"])
@pytest.mark.parametrize("fused", [False, True], ids=["eq2", "alg8"])
@pytest.mark.parametrize("halving", [False, True], ids=["fold", "halving"])
@pytest.mark.parametrize("log2n", ALL_LOG2N)
def test_polymul32_all_sizes(oracle, log2n, halving, fused, row_ops):
    """N = 2 .. 2^17: radix-2 kernel, single row, 2^13 one-CTA kernel and the
    column split; 2 polys x 3 limbs of 30-bit primes."""
    if fused and log2n < 2:
        pytest.skip("Algorithm 8 needs N >= 4")
    n = 1 << log2n
    L, P = (3, 2) if log2n <= 15 else (2, 1)
    plan, qs, psis = _plan(log2n, L, halving=halving, fused=fused, row_ops=row_ops)
    a, b = operands(60000 + log2n, qs, P, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    got = to_host32(plan.polymul(to_dev32(a), to_dev32(b)))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("row_ops", [1, 3, 4], ids=["rows1", "rowslat", "wide"])
@pytest.mark.parametrize("halving", [False, True], ids=["fold", "halving"])
@pytest.mark.parametrize("log2n", ALL_LOG2N)
def test_ntt32_fwd_inv_all_sizes(oracle, log2n, halving, row_ops):
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2, halving=halving,
                           row_ops=row_ops if log2n >= (10 if row_ops == 4 else 12) else None)
    x, y = operands(61000 + log2n, qs, 1, n)
    d = to_dev32(x)
    plan.ntt_fwd_(d)
    fwd = to_host32(d)
    for l in range(2):
        assert np.array_equal(fwd[0, l], oracle.ntt_fwd_bo(x[0, l], qs[l], psis[l])), l
    plan.ntt_inv_(d)
    assert np.array_equal(to_host32(d), x)
    d2 = to_dev32(y)
    plan.ntt_inv_(d2)
    inv = to_host32(d2)
    for l in range(2):
        assert np.array_equal(inv[0, l], oracle.ntt_inv_bo(y[0, l], qs[l], psis[l])), l


def test_pointwise32_extremes():
    """Algorithm 4 with 32-bit words at the edges, and the paper's Sec. IV-C
    example (q = 994705409, 994674970 * 994705408 mod q = 30439)."""
    from paper_2209_01290_gb300 import Plan
    q, log2n = 994705409, 4
    plan = Plan(1 << log2n, [q], word32=True)
    n = 1 << log2n
    vals = [0, 1, q - 1, q - 2, (q - 1) // 2, 2, q // 3]
    a = np.array([vals[i % len(vals)] for i in range(n)], dtype=np.uint64)
    b = np.array([vals[(i * 3 + 1) % len(vals)] for i in range(n)], dtype=np.uint64)
    a[0], b[0] = 994674970, 994705408
    got = to_host32(plan.pointwise(to_dev32(a), to_dev32(b)))
    assert got.tolist() == [(int(x) * int(y)) % q for x, y in zip(a, b)]
    assert int(got[0]) == 30439


@pytest.mark.parametrize("log2n", [3, 11, 12, 13, 16, 17])
def test_word32_edges(oracle, log2n):
    """Maximal words, monomials across the wrap, sampled schoolbook coefficients."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 1)
    q = qs[0]
    full = np.full((1, 1, n), q - 1, np.uint64)
    got = to_host32(plan.polymul(to_dev32(full), to_dev32(full)))
    assert np.array_equal(got[0, 0], np.array([(2 * k + 2 - n) % q for k in range(n)], np.uint64))
    rng = np.random.default_rng(log2n)
    for i, j in [(0, 0), (n - 1, n - 1), (n - 1, 1), tuple(rng.integers(0, n, 2))]:
        a = np.zeros((1, 1, n), np.uint64)
        b = np.zeros((1, 1, n), np.uint64)
        a[0, 0, i] = 1
        b[0, 0, j] = 1
        want = np.zeros(n, np.uint64)
        if i + j < n:
            want[i + j] = 1
        else:
            want[i + j - n] = q - 1
        assert np.array_equal(to_host32(plan.polymul(to_dev32(a), to_dev32(b)))[0, 0], want)
    a, b = operands(62000 + log2n, qs, 1, n)
    got = to_host32(plan.polymul(to_dev32(a), to_dev32(b)))
    for k in rng.integers(0, n, 4):
        assert int(got[0, 0, k]) == schoolbook_coeff(a[0, 0], b[0, 0], q, int(k))


def test_word32_paper_prime(oracle):
    """The paper's 30-bit prime 994705409 supports N = 2^16."""
    from paper_2209_01290_gb300 import Plan
    q, n = 994705409, 1 << 16
    plan = Plan(n, [q], word32=True)
    a, b = operands(63000, [q], 1, n)
    want = oracle.polymul_ntt(a[0, 0], b[0, 0], q, plan.psis[0])
    assert np.array_equal(to_host32(plan.polymul(to_dev32(a), to_dev32(b)))[0, 0], want)


@pytest.mark.parametrize("log2n", [12, 14, 16])
def test_word32_aliasing(oracle, log2n):
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2)
    a, b = operands(64000 + log2n, qs, 1, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    want_sq = oracle_polymul_batch(oracle, a, a, qs, psis)
    da, db = to_dev32(a), to_dev32(b)
    plan.polymul(da, db, out=da)
    assert np.array_equal(to_host32(da), want)
    da, db = to_dev32(a), to_dev32(b)
    plan.polymul(da, db, out=db)
    assert np.array_equal(to_host32(db), want)
    da = to_dev32(a)
    plan.polymul(da, da, out=da)
    assert np.array_equal(to_host32(da), want_sq)


def test_word32_checks():
    """Word-size rules of the C ABI: q < 2^30 for PM_PLAN_WORD32, 32-bit
    plans only through the *32 calls and the other way round, no persistent
    variant; pm_check_reduced32 sees an unreduced word."""
    import torch
    from paper_2209_01290_gb300 import Plan, capi
    qs60, psis60 = capi.pm_find_params(12, 1, 60)
    with pytest.raises(capi.PMError) as ei:
        Plan(1 << 12, qs60, psis60, word32=True)
    assert capi.STATUS_NAMES[ei.value.status] == "PM_ERR_Q"
    p32, qs, _ = _plan(12, 1)
    p64 = Plan(1 << 12, qs60, psis60)
    x32 = torch.zeros(1 << 12, dtype=torch.int32, device="cuda")
    x64 = torch.zeros(1 << 12, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.PMError):
        capi.pm_polymul(p32.handle, x64.data_ptr(), x64.data_ptr(), x64.data_ptr(), 1)
    with pytest.raises(capi.PMError):
        capi.pm_polymul32(p64.handle, x32.data_ptr(), x32.data_ptr(), x32.data_ptr(), 1)
    with pytest.raises(capi.PMError):
        capi.pm_plan_tune(p32.handle, capi.PM_VARIANT_PERSISTENT)
    with pytest.raises(TypeError):
        p32.polymul(x64, x64)
    a, _ = operands(65000, qs, 1, 1 << 12)
    d = to_dev32(a)
    assert p32.check_reduced(d)
    a[0, 0, 5] = qs[0]
    assert not p32.check_reduced(to_dev32(a))


def test_word32_batch_sampled(oracle):
    """A 64-product N=2^16 batch: sampled units in full against the oracle."""
    log2n, P, L = 16, 8, 8
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, L)
    a, b = operands(66000, qs, P, n)
    got = to_host32(plan.polymul(to_dev32(a), to_dev32(b)))
    rng = np.random.default_rng(2)
    for u in rng.choice(P * L, 3, replace=False):
        p, l = divmod(int(u), L)
        assert np.array_equal(got[p, l], oracle.polymul_ntt(a[p, l], b[p, l], qs[l], psis[l]))
