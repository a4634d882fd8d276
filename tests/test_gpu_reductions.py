"""The reduction variants of the Sec. II-B study, on the GPU, against exact
integer arithmetic (random operands and edge cases, 30/60/62-bit moduli),
including the paper's example a=994674970, b=994705408, q=994705409."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bits", [30, 60, 62])
@pytest.mark.parametrize("variant", range(6))
def test_reduction_variant(oracle, bits, variant):
    import torch
    from paper_2209_01290_gb300 import capi
    if variant == 2 and bits > 60:
        pytest.skip("Algorithm 3 needs len(q) <= 60")
    q = oracle.find_primes(1 << 4, 1, bits)[0]
    rng = np.random.default_rng(bits * 10 + variant)
    n = 1 << 16
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    edge = [0, 1, q - 1, q - 2, (q - 1) // 2, (q + 1) // 2]
    a[: len(edge) ** 2] = np.repeat(edge, len(edge))
    b[: len(edge) ** 2] = np.tile(edge, len(edge))
    da, db = to_dev(a), to_dev(b)
    dc = torch.empty_like(da)
    capi.pm_reduction_apply(variant, q, da.data_ptr(), db.data_ptr(), dc.data_ptr(), n)
    torch.cuda.synchronize()
    got = to_host(dc)
    want = [(int(x) * int(y)) % q for x, y in zip(a, b)]
    assert got.tolist() == want


def test_paper_example_all_variants():
    import torch
    from paper_2209_01290_gb300 import capi
    a, b, q = 994674970, 994705408, 994705409
    da = to_dev(np.array([a], np.uint64))
    db = to_dev(np.array([b], np.uint64))
    for v in range(6):
        dc = torch.empty_like(da)
        capi.pm_reduction_apply(v, q, da.data_ptr(), db.data_ptr(), dc.data_ptr(), 1)
        torch.cuda.synchronize()
        assert int(to_host(dc)[0]) == 30439, v


def test_reduction_rates_positive():
    from paper_2209_01290_gb300 import capi
    r = capi.pm_reduction_rates(0, 0xffffffffffc0001)
    assert all(v > 0 for v in r.values())
