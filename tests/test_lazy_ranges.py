"""Host check (no GPU) of the wide lazy ranges the 1024-word split uses for
60-bit primes (pm_arith.cuh, pm_wide.cuh, pm_passes.cuh), with the schedule
restated from the sources: interval arithmetic on value bounds (in units of
q) through every stage, for every column count CL = 1..7 (N = 2^11..2^17),
for Eq. 2 and for Algorithm 8's truncated transforms.

Rules checked at each step:
* a conditional subtraction of m needs its input below 2m;
* the forward CT butterfly (x + t, x - t + 2q) with t = Shoup(y) in [0, 2q)
  grows the bound by 2q; the GS difference x - y + 8q needs y < 8q;
* every value stays below 16q, which fits a 64-bit word for every prime
  q < 2^60 (the plan enables these ranges only then);
* Algorithm 4 gets operands below q (its REQUIRE x < 2^2m holds);
* the outputs are canonical after the last reduction.
"""

Q_MAX = (1 << 60) - 1  # any prime the wide ranges are enabled for is below 2^60
WORD = 1 << 64


def _fits(bound_q):
    # values are below bound_q * q <= bound_q * (2^60 - 1)
    assert bound_q * Q_MAX <= WORD, bound_q


def _csub(bound, m):
    """x < bound -> csub(x, m) < m (needs bound <= 2m)."""
    assert bound <= 2 * m, (bound, m)
    return m


def _ct(bound, reduce_by):
    """One CT butterfly with inputs below `bound` (q units): (a + t, a - t + 2)."""
    a = _csub(bound, reduce_by) if reduce_by else bound
    out = a + 2
    _fits(out)
    return out


def _gs(bound, reduce_sum):
    """One GS butterfly (m = 8q): s = x + y [csub 8], y' = Shoup(x - y + 8) < 2."""
    assert bound <= 8  # y < 8q keeps x - y + 8q positive
    _fits(bound + 8)  # the difference
    s = 2 * bound
    _fits(s)
    if reduce_sum:
        s = _csub(s, 8)
    return max(s, 2)


def _forward(cl, fused):
    b = 1  # canonical input
    for _ in range(cl):  # k_wcol_fwd with LZ: ct_col / ct_tail, RED = false
        b = _ct(b, 0)
    assert b <= 15
    b = 16  # the row kernel assumes only "below 16q" for its input
    stages = 9 if fused else 10  # Algorithm 8 omits the last forward stage
    for r in range(stages):  # w_fwd_pass: csub by 8q at in-row stages 0, 4, 8
        b = _ct(b, 8 if r % 4 == 0 else 0)
    return b


def _reduce16(bound):
    """reduce16: csub 8q, 4q, 2q, q."""
    assert bound <= 16
    b = bound
    for m in (8, 4, 2, 1):
        b = min(b, _csub(b, m))
    return b


def _inverse(cl, start_bound, first_stage):
    b = start_bound
    for r in range(first_stage, 10):  # w_inv_pass: sums reduced from r = 3 on
        b = _gs(b, r >= 3)
    for _ in range(cl - 1):  # k_wcol_inv with LZ: every sum reduced by 8q
        b = _gs(b, True)
    # the last stage folds 1/N: s = x + y, d = x - y + 8q, both Shoup
    assert b <= 8
    _fits(2 * b)
    _fits(b + 8)
    out = 2
    return _csub(out, 1)  # final csub to [0, q)


def test_eq2_ranges_all_column_counts():
    for cl in range(1, 8):
        fb = _forward(cl, fused=False)
        assert fb <= 16
        assert _reduce16(fb) == 1  # Algorithm 4 operands below q
        # the product is canonical; the inverse starts below q
        assert _inverse(cl, 1, 0) == 1


def test_algorithm8_ranges_all_column_counts():
    for cl in range(1, 8):
        fb = _forward(cl, fused=True)
        assert _reduce16(fb) == 1  # fused_pair reduces its four inputs
        # the pair step's outputs are brought to [0, 2q); the inverse then
        # skips its first stage
        assert _inverse(cl, 2, 1) == 1


def test_forward_ntt_output_canonical():
    for cl in range(0, 8):
        b = 1
        for _ in range(cl):
            b = _ct(b, 0)
        b = 16
        for r in range(10):
            b = _ct(b, 8 if r % 4 == 0 else 0)
        assert _reduce16(b) == 1


def test_headroom_needs_q_below_2_60():
    # 16q fits a word only for q <= 2^60: a 61-bit prime would overflow
    assert 16 * Q_MAX < WORD
    assert 16 * ((1 << 61) - 1) >= WORD
