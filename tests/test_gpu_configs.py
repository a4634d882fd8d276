"""The five workload configurations, bit-exact against the oracle.

C1 single N=2^12 product; C2 N=2^13..2^17 (forward, inverse, product);
C3 N=2^16 with the 32 largest 60-bit primes = 1 mod 2^17; C4 an uneven batch
(N and limb count drawn per job) computed in one call per job shape; C5's
request mix is covered by the serving tests."""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, to_dev, to_host
from paper_2209_01290_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_c1_single_4096(oracle):
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(12, 1, 60)
    assert qs[0] == 0xfffffffffffc001
    a, b = operands(inputs.seed_for(0), qs, 1, 1 << 12)
    got = to_host(Plan(1 << 12, qs, psis).polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got[0, 0], oracle.schoolbook(a[0, 0], b[0, 0], qs[0]))


@pytest.mark.parametrize("log2n", [13, 14, 15, 16, 17])
def test_c2_sweep(oracle, log2n):
    from paper_2209_01290_gb300 import Plan, capi
    n = 1 << log2n
    qs, psis = capi.pm_find_params(log2n, 1, 60)
    plan = Plan(n, qs, psis)
    a, b = operands(inputs.seed_for(1) + log2n, qs, 1, n)
    got = to_host(plan.polymul(to_dev(a), to_dev(b)))
    assert np.array_equal(got[0, 0], oracle.polymul_ntt(a[0, 0], b[0, 0], qs[0], psis[0]))
    d = to_dev(a)
    plan.ntt_fwd_(d)
    assert np.array_equal(to_host(d)[0, 0], oracle.ntt_fwd_bo(a[0, 0], qs[0], psis[0]))
    plan.ntt_inv_(d)
    assert np.array_equal(to_host(d), a)


def test_c3_rns_32_limbs(oracle):
    from paper_2209_01290_gb300 import Plan, capi
    log2n, L = 16, 32
    qs, psis = capi.pm_find_params(log2n, L, 60)
    assert len(set(qs)) == 32 and qs[-1] == 1152921504538951681
    plan = Plan(1 << log2n, qs, psis)
    a, b = operands(inputs.seed_for(2), qs, 1, 1 << log2n)
    want = oracle_polymul_batch(oracle, a, b, qs, psis)
    for variant in (1, 0):
        capi.pm_plan_tune(plan.handle, variant)
        assert np.array_equal(to_host(plan.polymul(to_dev(a), to_dev(b))), want), variant


def test_c4_uneven_sample(oracle):
    """A sample of the uneven batch: each job with its own N, limb count and
    largest primes; every job checked (full limbs for small jobs, sampled
    limbs for large ones)."""
    from paper_2209_01290_gb300 import Plan, capi
    shapes = inputs.uneven_shapes(inputs.seed_for(3), njobs=12)
    rng = np.random.default_rng(5)
    for j, sh in enumerate(shapes):
        n = 1 << sh.log2n
        L = min(sh.nlimbs, 6)
        qs, psis = capi.pm_find_params(sh.log2n, L, 60)
        plan = Plan(n, qs, psis)
        a, b = operands(inputs.seed_for(3) + 100 + j, qs, 1, n)
        got = to_host(plan.polymul(to_dev(a), to_dev(b)))
        for l in rng.choice(L, min(L, 2), replace=False):
            want = oracle.polymul_ntt(a[0, l], b[0, l], qs[l], psis[l])
            assert np.array_equal(got[0, l], want), (j, sh, l)
