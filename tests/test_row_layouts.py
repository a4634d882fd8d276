"""Host checks (no GPU) of the shared-memory layouts the row kernels use, with
the index formulas restated from the kernel sources:

* the radix-4 passes of a 1024-word row over 256 threads (pm_wide.cu) and of
  a 4096-word row over 1024 threads (k_rows_lat): every pass covers each
  word exactly once, and no access is bank-conflicted for 64-bit words
  (padding one word per 16, a half-warp per wavefront) or, for the 1024-word
  rows, for 32-bit words (one word per 32, a warp per wavefront);
* the twiddle slices a 1024-word row stages in shared memory: every entry of
  row t's in-row stages lands in its own slot, and the positions the passes
  read hold the entries Algorithm 6 / 7 index (Psi_br[2^s + t 2^r + i]);
* the bulk copies (TMA) that stage those slices for 64-bit words: each slice
  is one contiguous run of the table, both ends 16-byte aligned, the copies
  tile slots 0 .. 1022 exactly and leave slot 1023 (the mbarrier) alone.
"""


def _geo(LR, E, th, ef):
    """Thread th's group in the pass with stride 2^E: (its first word j0, blk)."""
    TB = LR - 2
    if E >= ef:
        off, blk = th & ((1 << E) - 1), th >> E
    else:
        blk, off = th & ((1 << (TB - E)) - 1), th >> (TB - E)
    return (blk << (E + 2)) + off, blk


def _pad(j, shift):
    return j + (j >> shift)


def _worst_ways(addrs, group):
    """Max accesses to one bank slot within any `group` consecutive threads
    (addresses in words of the bank width: 8 bytes x 16 slots or 4 x 32)."""
    worst = 0
    for base in range(0, len(addrs), group):
        banks = [a % group for a in addrs[base:base + group]]
        worst = max(worst, max(banks.count(b) for b in set(banks)))
    return worst


def _check_rows(LR, word_bytes, ef):
    T = 1 << (LR - 2)
    shift = 4 if word_bytes == 8 else 5
    group = 16 if word_bytes == 8 else 32
    for p in range(LR // 2):
        E = LR - 2 - 2 * p
        words = []
        for u in range(4):
            addrs = []
            for th in range(T):
                j0, _ = _geo(LR, E, th, ef)
                j = j0 + (u << E)
                words.append(j)
                addrs.append(_pad(j, shift))
            assert _worst_ways(addrs, group) == 1, (LR, word_bytes, p, u)
        assert sorted(words) == list(range(1 << LR)), (LR, p)


def test_wide_rows_64bit():
    _check_rows(10, 8, 4)


def test_wide_rows_32bit():
    _check_rows(10, 4, 5)


def test_latency_rows_64bit():
    _check_rows(12, 8, 4)


def _stage(LR, logn, t):
    """Slot -> global table index of row t's staged slices (w_stage_tw): slot
    i = 2^r - 1 + e holds entry e of slice r."""
    slots = {}
    for i in range((1 << LR) - 1):
        r = (i + 1).bit_length() - 1
        e = i + 1 - (1 << r)
        idx = (1 << (logn - LR + r)) + (t << r) + e
        slot = (1 << r) - 1 + e
        assert slot not in slots
        slots[slot] = idx
    return slots


def _bulk(LR, logn, t):
    """(smem slot, global index, entries) of each bulk copy of one table
    (w_stage_tw_bulk): slice r, 2^r entries."""
    return [((1 << r) - 1, (1 << (logn - LR + r)) + (t << r), 1 << r) for r in range(LR)]


def test_twiddle_slices_hold_the_indexed_entries():
    LR = 10
    for logn in (10, 13, 16, 17):
        N = 1 << logn
        for t in sorted({0, 1, (1 << (logn - LR)) - 1} & set(range(1 << (logn - LR)))):
            slots = _stage(LR, logn, t)
            assert sorted(slots) == list(range((1 << LR) - 1))
            assert all(0 <= v < N for v in slots.values())
            for p in range(LR // 2):
                E = LR - 2 - 2 * p
                for th in range(1 << (LR - 2)):
                    j0, blk = _geo(LR, E, th, 4)
                    # forward stage 2p: Psi_br[2^s + t 2^(2p) + blk], s = n-10+2p
                    s0 = logn - LR + 2 * p
                    assert slots[(1 << (2 * p)) - 1 + blk] == (1 << s0) + (t << (2 * p)) + blk
                    # stage 2p+1, pair u/2 = 0, 1: entries 2 blk, 2 blk + 1
                    base = (1 << (2 * p + 1)) - 1 + 2 * blk
                    for h, slot in enumerate((base, base + 1)):
                        want = (1 << (s0 + 1)) + (t << (2 * p + 1)) + 2 * blk + h
                        assert slots[slot] == want, (logn, t, p, th, h)


def test_bulk_copies_match_the_staged_slices():
    LR, TW = 10, 16  # 16-byte twiddle pairs (64-bit words)
    for logn in (10, 13, 16, 17):
        for t in sorted({0, 1, (1 << (logn - LR)) - 1} & set(range(1 << (logn - LR)))):
            slots = _stage(LR, logn, t)
            covered = []
            for slot, idx, cnt in _bulk(LR, logn, t):
                assert (slot * TW) % 16 == 0 and (idx * TW) % 16 == 0 and (cnt * TW) % 16 == 0
                for e in range(cnt):
                    assert slots[slot + e] == idx + e
                covered += range(slot, slot + cnt)
            assert sorted(covered) == list(range((1 << LR) - 1))
            assert (1 << LR) - 1 not in covered  # the mbarrier's slot
            assert sum(c for *_, c in _bulk(LR, logn, t)) * TW == ((1 << LR) - 1) * TW
