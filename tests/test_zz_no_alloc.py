"""The allocation-free product entry point (pm_polymul_noalloc), called
through the C ABI, must give exactly what pm_polymul gives.  This file sorts
last so that a stopping run has already run every other test; it also passes
on its own in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(capi, plan, fn, a, b):
    import torch
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    dc = torch.empty_like(da)
    s = torch.cuda.current_stream().cuda_stream
    fn(plan.handle, da.data_ptr(), db.data_ptr(), dc.data_ptr(), a.shape[0], s)
    torch.cuda.synchronize()
    return dc.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("log2n,nlimbs,npoly", [(16, 2, 8), (17, 1, 16), (14, 3, 2), (12, 2, 3)])
def test_noalloc_matches_polymul_twice(log2n, nlimbs, npoly):
    import torch
    assert torch.cuda.is_available()
    from paper_2209_01290_gb300 import Plan, capi, inputs
    n = 1 << log2n
    qs, psis = capi.pm_find_params(log2n, nlimbs, 60)
    plan = Plan(n, qs, psis)
    for call in range(2):  # two calls in a row share the static scratch
        a, b = inputs.operand_pair(inputs.seed_for(0) + 31 * call + log2n, qs, npoly, n)
        want = _run(capi, plan, capi.pm_polymul, a, b)
        got = _run(capi, plan, capi.pm_polymul_noalloc, a, b)
        assert np.array_equal(got, want), (log2n, call)
    plan.close()


def test_noalloc_scratch_bound():
    """Two distinct operands at N = 2^16 need scratch: 32 products (exactly
    2^21 words) run and match pm_polymul, 33 are rejected.  A square of the
    same 33 products keeps its one image in c and needs no scratch."""
    from paper_2209_01290_gb300 import Plan, capi, inputs
    import torch
    log2n = 16
    n = 1 << log2n
    qs, psis = capi.pm_find_params(log2n, 1, 60)
    plan = Plan(n, qs, psis)
    a, b = inputs.operand_pair(inputs.seed_for(0) + 977, qs, 32, n)
    want = _run(capi, plan, capi.pm_polymul, a, b)
    got = _run(capi, plan, capi.pm_polymul_noalloc, a, b)  # 32 * 2^16 = 2^21 words
    assert np.array_equal(got, want)
    npoly = 33  # 33 * 2^16 > 2^21 words
    da = torch.zeros((npoly, 1, n), dtype=torch.int64, device="cuda")
    db = torch.ones((npoly, 1, n), dtype=torch.int64, device="cuda")
    dc = torch.empty_like(da)
    with pytest.raises(capi.PMError) as e:
        capi.pm_polymul_noalloc(plan.handle, da.data_ptr(), db.data_ptr(), dc.data_ptr(),
                                npoly, 0)
    assert e.value.status == -1 and "2^21" in str(e.value)
    sq, _ = inputs.operand_pair(inputs.seed_for(0) + 978, qs, npoly, n)
    want = _run(capi, plan, capi.pm_polymul, sq, sq)
    ds = torch.from_numpy(sq.view(np.int64)).cuda()
    dq = torch.empty_like(ds)
    capi.pm_polymul_noalloc(plan.handle, ds.data_ptr(), ds.data_ptr(), dq.data_ptr(), npoly,
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(dq.cpu().numpy().view(np.uint64), want)
    plan.close()
