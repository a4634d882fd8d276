"""Host checks (no GPU) of the ticket orders of the persistent launches on
the 1024-word split (pm_wpersist.cu), with the index rules restated from the
sources:

* the compact lagged order of a uniform batch (k_wpersist): group g holds
  the column-forward tasks of unit g, the rows of unit g - lagF and the
  column-inverse tasks of unit g - lagI; groups fall into segments with the
  same set of tasks, so no ticket is empty.  Every task appears exactly once
  and a unit's rows come after all its column-forward tasks, its inverse
  tasks after all its rows (so every wait is for smaller tickets);
* the block tables of an uneven batch (k_wuneven): the unit of every ticket
  is found from the unit of the block's first ticket by a forward scan.
"""
import itertools

import numpy as np


def _segments(U, F, W, I, lagF, lagI):
    lagI = lagI if lagI > lagF else lagF + 1
    G = U + lagI
    bp = sorted([0, lagF, lagI, U, U + lagF, G])
    segs, t = [], 0
    for k in range(5):
        g0, g1 = bp[k], bp[k + 1]
        if g1 <= g0 or g0 >= G:
            continue
        m = (1 if g0 < U else 0) | (2 if lagF <= g0 < U + lagF else 0) | \
            (4 if lagI <= g0 < U + lagI else 0)
        gs = (F if m & 1 else 0) + (W if m & 2 else 0) + (I if m & 4 else 0)
        if gs == 0:
            continue
        segs.append((g0, t, m, gs))
        t += (g1 - g0) * gs
    return segs, t, lagI


def _decode(segs, t, F, W, lagF, lagI):
    k = 0
    while k + 1 < len(segs) and t >= segs[k + 1][1]:
        k += 1
    g0, t0, m, gs = segs[k]
    off = t - t0
    g, r = g0 + off // gs, off % gs
    if m & 1 and r < F:
        return ("f", g, r)
    if m & 1:
        r -= F
    if m & 2 and r < W:
        return ("w", g - lagF, r)
    if m & 2:
        r -= W
    return ("i", g - lagI, r)


def test_compact_lagged_order():
    # tasks per unit of the 1024-word split: F = 2 x tiles, W = 2^CL, I = tiles
    shapes = [(8, 8, 4), (16, 16, 8), (32, 64, 16), (64, 128, 32), (16, 64, 16)]
    for U, (F, W, I), lagF, lagI in itertools.product([1, 2, 5, 32, 100], shapes,
                                                     [1, 2, 8, 40], [2, 16, 32, 90]):
        segs, T, lI = _segments(U, F, W, I, lagF, lagI)
        assert len(segs) <= 8
        assert T == U * (F + W + I)  # no empty ticket
        pos = {}
        for t in range(T):
            task = _decode(segs, t, F, W, lagF, lI)
            assert task not in pos
            pos[task] = t
        assert len(pos) == T
        for u in range(U):
            f_last = max(pos[("f", u, r)] for r in range(F))
            w = [pos[("w", u, r)] for r in range(W)]
            i_first = min(pos[("i", u, r)] for r in range(I))
            assert f_last < min(w) and max(w) < i_first


def _wp_tiles(cl):
    return 32 if cl == 7 else (4 << (cl - 3)) if cl > 3 else 4


def test_uneven_block_tables():
    rng = np.random.default_rng(7)
    logns = rng.integers(12, 18, 300)
    squares = rng.random(300) < 0.2
    tasks = []
    for ln, sq in zip(logns, squares):
        cl = int(ln) - 10
        tasks.append(((1 if sq else 2) * _wp_tiles(cl), 1 << cl, _wp_tiles(cl)))
    for sec in range(3):
        counts = [t[sec] for t in tasks]
        assert max(sum(t) for t in tasks) <= 224  # at most 7 block entries per unit
        pre = np.concatenate([[0], np.cumsum(counts)[:-1]])
        total = int(sum(counts))
        blk, u = [], 0
        for i in range((total + 31) // 32):
            while u + 1 < len(pre) and pre[u + 1] <= 32 * i:
                u += 1
            blk.append(u)
        for x in range(total):
            v = blk[x >> 5]
            steps = 0
            while v + 1 < len(pre) and pre[v + 1] <= x:
                v += 1
                steps += 1
            assert pre[v] <= x < pre[v] + counts[v]
            assert steps <= 8
