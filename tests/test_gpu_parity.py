"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Every output word must equal the oracle's: the method is exact integer
arithmetic with canonical outputs in [0, q), so the tolerance is zero.
"""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, schoolbook_coeff, to_dev, to_host

pytestmark = pytest.mark.gpu

ALL_LOG2N = list(range(1, 18))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _plan(log2n, nlimbs, qbits=60, halving=False, variant=None):
    """variant: None (the plan's default launch) or (variant, row_ops)."""
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(log2n, nlimbs, qbits)
    plan = Plan(1 << log2n, qs, psis, halving=halving)
    if variant is not None:
        capi.pm_plan_tune(plan.handle, variant[0], row_ops=variant[1])
    return plan, qs, psis


VARIANTS = [(0, 1), (0, 2), (0, 3), (0, 4), (1, 1)]
VARIANT_IDS = ["split-rows1", "split-rows2", "split-rowslat", "split-wide", "persistent"]


@pytest.mark.parametrize("variant", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("halving", [False, True], ids=["fold1N", "halving"])
@pytest.mark.parametrize("log2n", ALL_LOG2N)
def test_polymul_all_sizes(torch_cuda, oracle, log2n, halving, variant):
    """Every code path: radix-2 smem kernel (N <= 2^11), single-row kernel
    (2^12), one-CTA 2^13 kernel, column split (2^14..2^17) as three launches
    (row kernel with the operands one after the other, together, or over
    1024 threads in radix-4 passes), the 1024-word-row split (N >= 2^10:
    one cluster launch up to 2^13) or one persistent work-queue launch
    (2^13..2^17); 2 polys x 3 limbs; 1/N folded into the last stage or
    applied as per-stage halving."""
    n = 1 << log2n
    L, P = (3, 2) if log2n <= 15 else (2, 1)
    plan, qs, psis = _plan(log2n, L, halving=halving, variant=variant)
    a, b = operands(1000 + log2n, qs, P, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    torch_cuda.cuda.synchronize()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("row_ops", [0, 1, 3, 4], ids=["auto", "rows1", "rowslat", "wide"])
@pytest.mark.parametrize("halving", [False, True], ids=["fold1N", "halving"])
@pytest.mark.parametrize("log2n", ALL_LOG2N)
def test_ntt_fwd_inv_all_sizes(torch_cuda, oracle, log2n, halving, row_ops):
    """Forward NTT equals the oracle's bo-order transform; inverse equals the
    oracle's inverse; inverse(forward(x)) = x.  Row kernels for N >= 4096:
    by batch size, 256 threads per row, 1024 threads per row; 1024-word rows
    for N >= 1024."""
    if row_ops and log2n < (10 if row_ops == 4 else 12):
        pytest.skip("no in-row kernel of this kind at this N")
    n = 1 << log2n
    L = 2
    plan, qs, psis = _plan(log2n, L, halving=halving, variant=(0, row_ops) if row_ops else None)
    x, y = operands(2000 + log2n, qs, 1, n)
    d = to_dev(x)
    plan.ntt_fwd_(d)
    fwd = to_host(d)
    for l in range(L):
        assert np.array_equal(fwd[0, l], oracle.ntt_fwd_bo(x[0, l], qs[l], psis[l])), l
    plan.ntt_inv_(d)
    assert np.array_equal(to_host(d), x)
    # inverse on an arbitrary bo-order vector
    d2 = to_dev(y)
    plan.ntt_inv_(d2)
    inv = to_host(d2)
    for l in range(L):
        assert np.array_equal(inv[0, l], oracle.ntt_inv_bo(y[0, l], qs[l], psis[l])), l


@pytest.mark.parametrize("log2n", [4, 12, 16])
def test_pointwise(torch_cuda, log2n):
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 3)
    a, b = operands(3000 + log2n, qs, 2, n)
    got = to_host(plan.pointwise(to_dev(a), to_dev(b)))
    for l, q in enumerate(qs):
        want = [(int(x) * int(y)) % q for x, y in zip(a[:, l].ravel(), b[:, l].ravel())]
        assert got[:, l].ravel().tolist() == want


def test_pointwise_extremes(torch_cuda):
    """Algorithm 4 at the edges: 0, 1, q-1, (q-1)^2, and the paper's example."""
    from paper_2209_01290_gb300 import Plan
    for q, log2n in [(0xffffffffffc0001, 4), (994705409, 4), (0x3fffffffffffffff, 1)]:
        import oracle as o
        if not o.is_prime(q) or (q - 1) % (2 << log2n):
            q = o.find_primes(1 << log2n, 1, q.bit_length())[0]
        plan = Plan(1 << log2n, [q])
        n = 1 << log2n
        vals = [0, 1, q - 1, q - 2, (q - 1) // 2, 2, q // 3]
        a = np.array([vals[i % len(vals)] for i in range(n)], dtype=np.uint64)
        b = np.array([vals[(i * 3 + 1) % len(vals)] for i in range(n)], dtype=np.uint64)
        if q == 994705409:
            a[0], b[0] = 994674970, 994705408
        got = to_host(plan.pointwise(to_dev(a), to_dev(b)))
        assert got.tolist() == [(int(x) * int(y)) % q for x, y in zip(a, b)]


@pytest.mark.parametrize("log2n", [3, 12, 13, 14, 16, 17])
def test_edge_inputs(torch_cuda, oracle, log2n):
    """Zeros, all q-1 (maximal words), monomials X^i * X^j (sign wrap)."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 1)
    q = qs[0]
    z = np.zeros((1, 1, n), np.uint64)
    full = np.full((1, 1, n), q - 1, np.uint64)
    got = to_host(plan.polymul(to_dev(z), to_dev(full)))
    assert not got.any()
    got = to_host(plan.polymul(to_dev(full), to_dev(full)))
    # (q-1)^2 * sum_{i,j} X^{i+j}: c_k = (k+1) - (N-1-k) = 2k + 2 - N
    want = np.array([(2 * k + 2 - n) % q for k in range(n)], dtype=np.uint64)
    assert np.array_equal(got[0, 0], want)
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
        assert np.array_equal(to_host(plan.polymul(to_dev(a), to_dev(b)))[0, 0], want), (i, j)


@pytest.mark.parametrize("log2n", [12, 13, 14, 16, 17])
def test_aliasing(torch_cuda, oracle, log2n):
    """c may alias a or b; a == b (squaring) also works."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2)
    a, b = operands(4000 + log2n, qs, 1, n)
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


@pytest.mark.parametrize("qbits,log2n", [(62, 12), (62, 16), (30, 12), (30, 16), (40, 14)])
def test_other_word_sizes(torch_cuda, oracle, qbits, log2n):
    """62-bit (Algorithm 4's limit for 64-bit words) and 30-bit moduli."""
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 2, qbits)
    a, b = operands(5000 + qbits + log2n, qs, 1, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    assert np.array_equal(to_host(plan.polymul(to_dev(a), to_dev(b))), want)


def test_paper_prime_994705409(torch_cuda, oracle):
    """The 30-bit prime of the paper's Barrett example supports N = 2^16."""
    from paper_2209_01290_gb300 import Plan
    q, n = 994705409, 1 << 16
    plan = Plan(n, [q])
    psi = plan.psis[0]
    assert psi == oracle.find_psi(q, n)
    a, b = operands(6000, [q], 1, n)
    want = oracle.polymul_ntt(a[0, 0], b[0, 0], q, psi)
    assert np.array_equal(to_host(plan.polymul(to_dev(a), to_dev(b)))[0, 0], want)


def test_given_psi_changes_ntt_not_product(torch_cuda, oracle):
    """The NTT depends on psi, the product does not."""
    from paper_2209_01290_gb300 import Plan, capi
    log2n = 14
    n = 1 << log2n
    qs, psis = capi.pm_find_params(log2n, 1, 60)
    q = qs[0]
    alt = pow(psis[0], 3, q)  # psi^3 is also a primitive 2N-th root
    p1, p2 = Plan(n, qs, psis), Plan(n, qs, [alt])
    a, b = operands(6100, qs, 1, n)
    c1 = to_host(p1.polymul(to_dev(a), to_dev(b)))
    c2 = to_host(p2.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(c1, c2)
    d = to_dev(a)
    p2.ntt_fwd_(d)
    assert np.array_equal(to_host(d)[0, 0], oracle.ntt_fwd_bo(a[0, 0], q, alt))


def test_check_reduced(torch_cuda):
    plan, qs, psis = _plan(12, 2)
    a, _ = operands(7000, qs, 1, 1 << 12)
    assert plan.check_reduced(to_dev(a))
    a[0, 1, 77] = qs[1]
    assert not plan.check_reduced(to_dev(a))


@pytest.mark.parametrize("log2n", [12, 16])
def test_polymul_host_pipeline(torch_cuda, oracle, log2n):
    """Host buffers in and out, copies pipelined in chunks."""
    import torch
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 3)
    P = 5
    a, b = operands(8000 + log2n, qs, P, n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    ha = torch.from_numpy(a.view(np.int64)).pin_memory()
    hb = torch.from_numpy(b.view(np.int64)).pin_memory()
    hc = torch.empty_like(ha).pin_memory()
    da, db, dc = (torch.empty(ha.shape, dtype=torch.int64, device="cuda") for _ in range(3))
    plan.polymul_host(ha, hb, hc, da, db, dc)
    assert np.array_equal(hc.numpy().view(np.uint64), want)


def test_streams_and_large_batch_sampled(torch_cuda, oracle):
    """A 64-product N=2^16 batch on a side stream; sampled units checked in
    full against the oracle and sampled coefficients against the definition."""
    import torch
    log2n, P, L = 16, 8, 8
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, L)
    a, b = operands(9000, qs, P, n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        da, db = to_dev(a), to_dev(b)
        dc = plan.polymul(da, db, stream=s)
    s.synchronize()
    got = to_host(dc)
    rng = np.random.default_rng(1)
    for u in rng.choice(P * L, 3, replace=False):
        p, l = divmod(int(u), L)
        want = oracle.polymul_ntt(a[p, l], b[p, l], qs[l], psis[l])
        assert np.array_equal(got[p, l], want), (p, l)
    for _ in range(4):
        p, l, k = int(rng.integers(P)), int(rng.integers(L)), int(rng.integers(n))
        assert int(got[p, l, k]) == schoolbook_coeff(a[p, l], b[p, l], qs[l], k)


@pytest.mark.slow
@pytest.mark.parametrize("row_ops", [0, 2], ids=["default", "rows4096"])
def test_headline_batch_sampled(torch_cuda, oracle, row_ops):
    """The benchmark's own workload and launch: 4096 products of N=2^16 with
    the largest 60-bit prime in one pm_polymul (default tuning: the
    1024-word split; also the 4096-word split).  Sampled units are checked in
    full against the oracle, sampled coefficients against the definition,
    and every output word is checked to be reduced."""
    from paper_2209_01290_gb300 import inputs
    log2n, P = 16, 4096
    n = 1 << log2n
    plan, qs, psis = _plan(log2n, 1, variant=(0, row_ops) if row_ops else None)
    da = inputs.uniform_limbs_torch(inputs.seed_for(9), qs, P, n)
    db = inputs.uniform_limbs_torch(inputs.seed_for(9) + 1, qs, P, n)
    dc = plan.polymul(da, db)
    torch_cuda.cuda.synchronize()
    assert plan.check_reduced(dc)
    rng = np.random.default_rng(16)
    for p in [0, P - 1] + [int(x) for x in rng.choice(np.arange(1, P - 1), 2, replace=False)]:
        a, b = to_host(da[p, 0]), to_host(db[p, 0])
        assert np.array_equal(to_host(dc[p, 0]), oracle.polymul_ntt(a, b, qs[0], psis[0])), p
    for _ in range(3):
        p, k = int(rng.integers(P)), int(rng.integers(n))
        got = int(to_host(dc[p, 0, k:k + 1])[0])
        assert got == schoolbook_coeff(to_host(da[p, 0]), to_host(db[p, 0]), qs[0], k)
