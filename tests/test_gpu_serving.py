"""The continuous-batching request loop (pm_server_*): every result is the
same as the product computed alone, under a budget tight enough that
requests wait for admission while others run."""
import threading

import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, to_dev, to_host

pytestmark = pytest.mark.gpu


class _DeviceView:
    """A CUDA-array-interface view of library-owned device memory."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<i8",
                                         "data": (ptr, False), "version": 3, "strides": None}


def _copy_out(ptr, shape):
    """Copy a server output (arena memory) into a fresh tensor."""
    import torch
    return torch.as_tensor(_DeviceView(ptr, shape), device="cuda").clone()


@pytest.mark.parametrize("budget_mb,inflight", [(2048, 2), (24, 2), (24, 1)])
def test_server_mix_equals_alone(oracle, budget_mb, inflight):
    """40 requests of mixed N (2^10 .. 2^16), limb counts and batch sizes
    (some squares), submitted from another thread.  Every result equals the
    product computed alone and the oracle's product.  The 24 MiB budget makes
    requests wait for admission while others run.  With two slots and no
    launch threshold (min_batch_rows 1) the device intervals of at least two
    batches overlap (timing events around each launch); with one slot they
    never do."""
    import torch
    from paper_2209_01290_gb300 import Plan, capi
    shapes = [(13, 3), (15, 1), (16, 2), (12, 4), (10, 2), (16, 1), (14, 2)]
    plans = {}
    for log2n, L in shapes:
        qs, psis = capi.pm_find_params(log2n, L, 60)
        plans[(log2n, L)] = (Plan(1 << log2n, qs, psis), qs, psis)
    rng = np.random.default_rng(budget_mb + inflight)
    reqs = []
    for i in range(40):
        # a heavy request first: it is still on the device when the next
        # batch launches
        log2n, L = (16, 2) if i == 0 else shapes[int(rng.integers(len(shapes)))]
        plan, qs, psis = plans[(log2n, L)]
        P = 4 if i == 0 else int(rng.integers(1, 3))
        a, b = operands(30000 + i, qs, P, 1 << log2n)
        if i % 7 == 3:
            b = a  # a square
        da = to_dev(a)
        db = da if i % 7 == 3 else to_dev(b)
        alone = plan.polymul(da, db)
        reqs.append((plan, da, db, P, alone, a, b, qs, psis))
    torch.cuda.synchronize()
    srv = capi.pm_server_create(0, budget_mb << 20, 0, inflight, min_batch_rows=1)
    ids = [None] * len(reqs)

    def producer():
        for i, (plan, da, db, P, *_rest) in enumerate(reqs):
            ids[i] = capi.pm_server_submit(srv, plan.handle, da.data_ptr(), db.data_ptr(), P)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    outs = []
    for i, (plan, da, db, P, alone, *_rest) in enumerate(reqs):
        ptr, lat = capi.pm_server_wait(srv, ids[i])
        assert lat > 0
        got = _copy_out(ptr, alone.shape)
        assert torch.equal(got, alone), i
        outs.append(to_host(got))
        capi.pm_server_release(srv, ids[i])
    st = capi.pm_server_get_stats(srv)
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["arena_used_bytes"] == 0
    assert st["arena_peak_bytes"] <= budget_mb << 20
    if budget_mb >= 2048:
        assert st["batches"] < len(reqs)  # requests were batched together
    assert st["max_inflight"] <= inflight
    if inflight >= 2:
        assert st["max_device_overlap"] >= 2, st  # batches overlapped on the device
    else:
        assert st["max_device_overlap"] == 1, st
    capi.pm_server_destroy(srv)
    # every result is the oracle's product
    for i, (plan, da, db, P, alone, a, b, qs, psis) in enumerate(reqs):
        want = oracle_polymul_batch(oracle, a, b, qs, psis)
        assert np.array_equal(outs[i], want), i


def test_server_budget_rejects_oversized():
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(16, 4, 60)
    plan = Plan(1 << 16, qs, psis)
    d = to_dev(np.zeros((8, 4, 1 << 16), np.uint64))
    srv = capi.pm_server_create(0, 8 << 20, 0, 2)  # 8 MiB: the 8x4x2^16 request cannot fit
    e = d[:1].clone()
    with pytest.raises(capi.PMError) as ex:
        capi.pm_server_submit(srv, plan.handle, d.data_ptr(), e.data_ptr(), 8)
    assert ex.value.status == -8
    capi.pm_server_destroy(srv)


def test_server_stop_with_arena_held():
    """Destroying a server whose queued request cannot fit beside the
    outputs the client still holds fails that request instead of waiting
    for releases that never come: destroy returns promptly."""
    import time
    from paper_2209_01290_gb300 import Plan, capi
    qs, psis = capi.pm_find_params(16, 1, 60)
    plan = Plan(1 << 16, qs, psis)
    a, b = operands(81000, qs, 4, 1 << 16)
    da, db = to_dev(a), to_dev(b)
    # 8 MiB: each request holds a 2 MiB output (plus 2 MiB of scratch while
    # it runs); three held outputs leave no room for a fourth request
    srv = capi.pm_server_create(0, 8 << 20, 0, 1)
    for _ in range(3):
        rid = capi.pm_server_submit(srv, plan.handle, da.data_ptr(), db.data_ptr(), 4)
        capi.pm_server_wait(srv, rid)
    stuck = capi.pm_server_submit(srv, plan.handle, da.data_ptr(), db.data_ptr(), 4)
    with pytest.raises(capi.PMError) as ex:
        capi.pm_server_wait(srv, stuck, timeout_ms=200)
    assert ex.value.status == -7
    t0 = time.time()
    capi.pm_server_destroy(srv)
    assert time.time() - t0 < 10
