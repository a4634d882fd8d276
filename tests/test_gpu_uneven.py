"""Uneven batches in one persistent launch (pm_polymul_uneven): products of
different N and limb counts, aliasing, and checks against the oracle."""
import numpy as np
import pytest

from helpers import operands, oracle_polymul_batch, to_dev, to_host
from paper_2209_01290_gb300 import inputs

pytestmark = pytest.mark.gpu


def _plans(shapes, halving=False):
    from paper_2209_01290_gb300 import Plan, capi
    cache = {}
    out = []
    for log2n, L in shapes:
        key = (log2n, L)
        if key not in cache:
            qs, psis = capi.pm_find_params(log2n, L, 60)
            cache[key] = (Plan(1 << log2n, qs, psis, halving=halving), qs, psis)
        out.append(cache[key])
    return out


MODES = [0, 1, 2]
MODE_IDS = ["auto", "persistent", "grouped"]


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_uneven_mixed_sizes(oracle, mode):
    from paper_2209_01290_gb300 import Queue
    shapes = [(12, 3), (17, 1), (13, 2), (3, 2), (16, 2), (14, 4), (15, 1), (12, 1), (16, 1)]
    plans = _plans(shapes)
    q = Queue(mode=mode)
    jobs, data = [], []
    for j, ((plan, qs, psis), (log2n, L)) in enumerate(zip(plans, shapes)):
        P = 2 if log2n <= 14 else 1
        a, b = operands(20000 + j, qs, P, 1 << log2n)
        da, db = to_dev(a), to_dev(b)
        dc = da.new_empty(da.shape)
        jobs.append((plan, da, db, dc))
        data.append((a, b, qs, psis, dc))
    for rep in range(2):  # the queue's buffers are reused
        q.polymul_uneven(jobs)
        q.sync()
        for a, b, qs, psis, dc in data:
            assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis))


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_uneven_aliasing(oracle, mode):
    from paper_2209_01290_gb300 import Queue
    shapes = [(14, 2), (16, 1), (13, 2), (12, 2)]
    plans = _plans(shapes)
    q = Queue(mode=mode)
    jobs, checks = [], []
    for j, ((plan, qs, psis), (log2n, L)) in enumerate(zip(plans, shapes)):
        a, b = operands(21000 + j, qs, 1, 1 << log2n)
        da, db = to_dev(a), to_dev(b)
        kind = j % 4
        if kind == 0:    # c = a
            jobs.append((plan, da, db, da)); checks.append((da, a, b, qs, psis))
        elif kind == 1:  # c = b
            jobs.append((plan, da, db, db)); checks.append((db, a, b, qs, psis))
        elif kind == 2:  # a = b = c (square in place)
            jobs.append((plan, da, da, da)); checks.append((da, a, a, qs, psis))
        else:            # square into a new buffer
            dc = da.new_empty(da.shape)
            jobs.append((plan, da, da, dc)); checks.append((dc, a, a, qs, psis))
    q.polymul_uneven(jobs)
    q.sync()
    for dc, a, b, qs, psis in checks:
        assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis))


def test_uneven_rejects_mixed_halving():
    from paper_2209_01290_gb300 import Queue, capi
    (p1, qs1, _), = _plans([(14, 1)])
    (p2, qs2, _), = _plans([(15, 1)], halving=True)
    a1 = to_dev(np.zeros((1, 1, 1 << 14), np.uint64))
    a2 = to_dev(np.zeros((1, 1, 1 << 15), np.uint64))
    with pytest.raises(capi.PMError) as e:
        Queue().polymul_uneven([(p1, a1, a1, a1), (p2, a2, a2, a2)])
    assert e.value.status == -1


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_uneven_halving_plans(oracle, mode):
    from paper_2209_01290_gb300 import Queue
    shapes = [(13, 1), (17, 1), (12, 2)]
    plans = _plans(shapes, halving=True)
    jobs, data = [], []
    for j, ((plan, qs, psis), (log2n, L)) in enumerate(zip(plans, shapes)):
        a, b = operands(22000 + j, qs, 1, 1 << log2n)
        da, db = to_dev(a), to_dev(b)
        dc = da.new_empty(da.shape)
        jobs.append((plan, da, db, dc))
        data.append((a, b, qs, psis, dc))
    q = Queue(mode=mode)
    q.polymul_uneven(jobs)
    q.sync()
    for a, b, qs, psis, dc in data:
        assert np.array_equal(to_host(dc), oracle_polymul_batch(oracle, a, b, qs, psis))


def test_uneven_mode_checks():
    from paper_2209_01290_gb300 import Queue, capi
    q = Queue()
    for bad in (-1, 3):
        with pytest.raises(capi.PMError):
            capi.pm_queue_set_mode(q._h, bad)


@pytest.mark.slow
@pytest.mark.parametrize("mode", [1, 2], ids=["persistent", "grouped"])
def test_c4_full_uneven_batch_sampled(oracle, mode):
    """The full uneven configuration: 512 jobs, N uniform over 2^12..2^17,
    1..48 limbs (the largest primes = 1 mod 2N), inputs generated on the
    device; one launch; 24 sampled (job, limb) units checked in full against
    the oracle."""
    import torch
    from paper_2209_01290_gb300 import Plan, Queue, capi
    shapes = inputs.uneven_shapes(inputs.seed_for(3), njobs=512)
    plans = {}
    jobs, meta = [], []
    for j, sh in enumerate(shapes):
        key = (sh.log2n, sh.nlimbs)
        if key not in plans:
            qs, psis = capi.pm_find_params(sh.log2n, sh.nlimbs, 60)
            plans[key] = (Plan(1 << sh.log2n, qs, psis), qs, psis)
        plan, qs, psis = plans[key]
        a = inputs.uniform_limbs_torch(inputs.seed_for(3) + 2 * j, qs, 1, 1 << sh.log2n)
        b = inputs.uniform_limbs_torch(inputs.seed_for(3) + 2 * j + 1, qs, 1, 1 << sh.log2n)
        c = torch.empty_like(a)
        jobs.append((plan, a, b, c))
        meta.append((qs, psis))
    q = Queue(mode=mode)
    q.polymul_uneven(jobs)
    q.sync()
    rng = np.random.default_rng(9)
    for j in rng.choice(len(jobs), 24, replace=False):
        plan, a, b, c = jobs[j]
        qs, psis = meta[j]
        l = int(rng.integers(len(qs)))
        want = oracle.polymul_ntt(to_host(a)[0, l], to_host(b)[0, l], qs[l], psis[l])
        assert np.array_equal(to_host(c)[0, l], want), (j, l)
