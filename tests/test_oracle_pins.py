"""Pins for the CPU oracle (no GPU).

Each test ties an oracle routine to something other than itself: hand-worked
fixtures (tests/golden), library routines (sympy number theory, numpy object
convolution, Python integers), closed forms, algebraic identities and brute
force.  Together they make a dropped term, a wrong sign or index or a swapped
operand in any oracle routine fail at least one test (see
test_oracle_mutants.py, which plants such mistakes and checks they are caught).
"""
import os
import random

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# small NTT-friendly primes: q = 1 mod 2N for the N used with them
SMALL_PRIMES = [17, 97, 7681, 12289, 40961, 65537, 786433]


def _fixture_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([list(map(int, part.split())) for part in line.split("|")])
    return rows


def _negacyclic_numpy(a, b, q):
    """Library route: full product by numpy convolution on Python ints, then
    fold with X^N = -1."""
    n = len(a)
    p = np.convolve(np.array([int(x) for x in a], dtype=object),
                    np.array([int(x) for x in b], dtype=object))
    c = [int(p[k]) - (int(p[k + n]) if k + n < len(p) else 0) for k in range(n)]
    return [x % q for x in c]


def _rand(rng_, n, q):
    return np.array([rng_.randrange(q) for _ in range(n)], dtype=np.uint64)


# ------------------------------------------------------------- fixtures ---
def test_golden_negacyclic_by_hand(oracle):
    for (n, q), a, b, c in _fixture_rows("negacyclic_small.txt"):
        assert len(a) == n
        assert oracle.schoolbook(a, b, q).tolist() == c
        psi = oracle.find_psi(q, n)
        assert oracle.polymul_ntt(a, b, q, psi).tolist() == c
        assert oracle.polymul_eq2(a, b, q, psi).tolist() == c
        if n >= 4:
            assert oracle.polymul_alg8(a, b, q, psi).tolist() == c


def test_golden_ntt_bo_by_hand(oracle):
    for (n, q, psi), a, ahat in _fixture_rows("ntt_bo_small.txt"):
        assert oracle.find_psi(q, n) == psi
        assert oracle.ntt_fwd_bo(a, q, psi, closed=True).tolist() == ahat
        assert oracle.ntt_fwd_bo(a, q, psi).tolist() == ahat
        assert oracle.ntt_inv_bo(ahat, q, psi, closed=True).tolist() == a
        assert oracle.ntt_inv_bo(ahat, q, psi).tolist() == a


def test_golden_barrett_example(oracle):
    (a, b, q), (want,) = _fixture_rows("barrett_example.txt")[0]
    import sympy
    assert sympy.isprime(q)
    assert oracle.is_prime(q)
    assert oracle.mulmod(a, b, q) == want
    x = a * b
    for alg in (2, 3, 4):
        r, k = oracle.barrett(alg, x, q)
        assert r == want, alg
    # Algorithms 3 and 4 take at most one correction (Sec. II-B)
    assert oracle.barrett(4, x, q)[1] <= 1
    assert oracle.barrett(3, x, q)[1] <= 1
    # q - 1 = 2^17 * 7589: an NTT prime for N up to 2^16
    assert (q - 1) % (1 << 17) == 0


# ------------------------------------------------------------- arithmetic ---
def test_mulmod_powmod_vs_python_ints(oracle):
    r = random.Random(1)
    for _ in range(2000):
        q = r.randrange(3, 1 << 62) | 1
        a, b = r.randrange(1 << 64), r.randrange(1 << 64)
        assert oracle.mulmod(a, b, q) == (a * b) % q
        e = r.randrange(1 << 64)
        assert oracle.powmod(a, e, q) == pow(a, e, q)


def test_half_rule(oracle):
    r = random.Random(2)
    for q in SMALL_PRIMES + [1152921504606830593]:
        for _ in range(500):
            x = r.randrange(q)
            h = oracle.half(x, q)
            assert 0 <= h < q and (2 * h) % q == x


def test_bitrev_brute(oracle):
    for bits in range(0, 12):
        for i in range(1 << bits):
            s = format(i, f"0{bits}b") if bits else ""
            assert oracle.bitrev(i, bits) == (int(s[::-1], 2) if bits else 0)


# ------------------------------------------------------------ setup ---------
@pytest.mark.parametrize("log2n", [12, 13, 14, 15, 16, 17])
def test_largest_prime_vs_sympy(oracle, log2n):
    import sympy
    n = 1 << log2n
    q = oracle.find_primes(n, 1, 60)[0]
    assert q < (1 << 60) and (q - 1) % (2 * n) == 0 and sympy.isprime(q)
    # no larger prime of that form below 2^60
    c = q + 2 * n
    while c < (1 << 60):
        assert not sympy.isprime(c)
        c += 2 * n


def test_prime_lists_vs_sympy(oracle):
    import sympy
    n = 1 << 16
    qs = oracle.find_primes(n, 32, 60)
    assert len(qs) == 32 and len(set(qs)) == 32
    assert qs == sorted(qs, reverse=True)
    # enumerate every candidate from 2^60 down to the 32nd prime with sympy
    want, c = [], ((1 << 60) - 2) // (2 * n) * (2 * n) + 1
    while len(want) < 32:
        if sympy.isprime(c):
            want.append(c)
        c -= 2 * n
    assert qs == want
    n17 = 1 << 17
    q17 = oracle.find_primes(n17, 48, 60)
    assert len(q17) == 48 and all(sympy.isprime(q) and q > (1 << 59) for q in q17)


def test_is_prime_vs_sympy(oracle):
    import sympy
    r = random.Random(3)
    for _ in range(3000):
        x = r.randrange(1 << 64)
        assert oracle.is_prime(x) == sympy.isprime(x)
    for p in SMALL_PRIMES:
        assert oracle.is_prime(p)
    # strong pseudoprimes to several small bases
    for c in [3215031751, 2152302898747, 3474749660383, 341550071728321,
              3825123056546413051]:
        assert not oracle.is_prime(c) and not sympy.isprime(c)


@pytest.mark.parametrize("q,log2n", [(17, 1), (17, 2), (17, 3), (97, 4), (7681, 8),
                                     (12289, 11), (1152921504606830593, 12),
                                     (994705409, 16)])
def test_psi_is_primitive_2n_root(oracle, q, log2n):
    import sympy
    n = 1 << log2n
    psi = oracle.find_psi(q, n)
    assert psi != 0 and sympy.n_order(psi, q) == 2 * n


# ------------------------------------------------------- polymul pins ------
@pytest.mark.parametrize("n", [2, 4, 8, 16, 64])
def test_schoolbook_vs_numpy_convolution(oracle, n):
    r = random.Random(n)
    for q in [17, 97, 7681, 1152921504606830593, (1 << 62) - 57]:
        if q < 1 << 20 and (q - 1) % (2 * n):
            continue
        a, b = _rand(r, n, q), _rand(r, n, q)
        assert oracle.schoolbook(a, b, q).tolist() == _negacyclic_numpy(a, b, q)


def test_schoolbook_exhaustive_n2_q17(oracle):
    q = 17
    for a0 in range(q):
        for a1 in range(0, q, 3):
            for b0 in range(0, q, 2):
                for b1 in range(q):
                    want = [(a0 * b0 - a1 * b1) % q, (a0 * b1 + a1 * b0) % q]
                    assert oracle.schoolbook([a0, a1], [b0, b1], q).tolist() == want


@pytest.mark.parametrize("n", [4, 16, 256])
def test_monomials(oracle, n):
    """X^i * X^j = X^{i+j}, or -X^{i+j-N} when i+j >= N (X^N = -1)."""
    q = 7681 if n <= 256 else 12289
    psi = oracle.find_psi(q, n)
    r = random.Random(n)
    for _ in range(20):
        i, j = r.randrange(n), r.randrange(n)
        a = np.zeros(n, np.uint64); a[i] = 1
        b = np.zeros(n, np.uint64); b[j] = 1
        want = np.zeros(n, np.uint64)
        if i + j < n:
            want[i + j] = 1
        else:
            want[i + j - n] = q - 1
        for f in (oracle.schoolbook,):
            assert f(a, b, q).tolist() == want.tolist()
        assert oracle.polymul_ntt(a, b, q, psi).tolist() == want.tolist()
        assert oracle.polymul_eq2(a, b, q, psi).tolist() == want.tolist()
        assert oracle.polymul_alg8(a, b, q, psi).tolist() == want.tolist()


def test_commutative_identity_linear(oracle):
    n, q = 64, 1152921504606830593
    r = random.Random(7)
    a, b, d = _rand(r, n, q), _rand(r, n, q), _rand(r, n, q)
    ab = oracle.schoolbook(a, b, q)
    assert ab.tolist() == oracle.schoolbook(b, a, q).tolist()
    one = np.zeros(n, np.uint64); one[0] = 1
    assert oracle.schoolbook(a, one, q).tolist() == a.tolist()
    bd = [(int(x) + int(y)) % q for x, y in zip(b, d)]
    lhs = oracle.schoolbook(a, bd, q).tolist()
    rhs = [(int(x) + int(y)) % q for x, y in zip(ab, oracle.schoolbook(a, d, q))]
    assert lhs == rhs


@pytest.mark.parametrize("n", [2, 8, 32])
def test_cyclic_ntt_vs_dft_definition(oracle, n):
    """NTT_omega(x)_j = sum_i x_i omega^{ij} (Sec. III-A), with Python ints."""
    q = 7681
    psi = oracle.find_psi(q, n)
    omega = psi * psi % q
    r = random.Random(n)
    x = _rand(r, n, q)
    want = [sum(int(x[i]) * pow(omega, i * j, q) for i in range(n)) % q for j in range(n)]
    assert oracle.ntt_cyclic(x, q, omega).tolist() == want


@pytest.mark.parametrize("log2n", [1, 3, 6, 10, 12])
def test_ntt_roundtrip_and_convolution_theorem(oracle, log2n):
    n = 1 << log2n
    q = oracle.find_primes(n, 1, 60)[0]
    psi = oracle.find_psi(q, n)
    omega = psi * psi % q
    r = random.Random(log2n)
    a, b = _rand(r, n, q), _rand(r, n, q)
    # INTT(NTT(a)) = a with the inverse (1/N) NTT_{omega^{-1}}
    fa = oracle.ntt_cyclic(a, q, omega)
    back = oracle.ntt_cyclic(fa, q, pow(omega, q - 2, q))
    ninv = pow(n, q - 2, q)
    assert [(int(v) * ninv) % q for v in back] == a.tolist()
    # cyclic convolution theorem, checked at small N against numpy's convolution
    if n <= 64:
        p = np.convolve(np.array([int(v) for v in a], dtype=object),
                        np.array([int(v) for v in b], dtype=object))
        cyc = [(int(p[k]) + (int(p[k + n]) if k + n < len(p) else 0)) % q for k in range(n)]
        fb = oracle.ntt_cyclic(b, q, omega)
        prod = np.array([(int(x) * int(y)) % q for x, y in zip(fa, fb)], dtype=np.uint64)
        got = oracle.ntt_cyclic(prod, q, pow(omega, q - 2, q))
        assert [(int(v) * ninv) % q for v in got] == cyc


@pytest.mark.parametrize("log2n", [1, 2, 5, 8, 10])
def test_polymul_ntt_vs_schoolbook(oracle, log2n):
    n = 1 << log2n
    for q in oracle.find_primes(n, 2, 60) + [oracle.find_primes(n, 1, 62)[0],
                                              oracle.find_primes(n, 1, 30)[0]]:
        psi = oracle.find_psi(q, n)
        r = random.Random(q)
        a, b = _rand(r, n, q), _rand(r, n, q)
        sb = oracle.schoolbook(a, b, q)
        assert oracle.polymul_ntt(a, b, q, psi).tolist() == sb.tolist()
        assert oracle.polymul_eq2(a, b, q, psi).tolist() == sb.tolist()
        if n >= 4:
            assert oracle.polymul_alg8(a, b, q, psi).tolist() == sb.tolist()


@pytest.mark.slow
def test_polymul_ntt_vs_schoolbook_4096(oracle):
    n = 4096
    q = oracle.find_primes(n, 1, 60)[0]
    psi = oracle.find_psi(q, n)
    r = random.Random(4096)
    a, b = _rand(r, n, q), _rand(r, n, q)
    assert oracle.polymul_ntt(a, b, q, psi).tolist() == oracle.schoolbook(a, b, q).tolist()


@pytest.mark.parametrize("log2n", [1, 2, 4, 7, 9])
def test_ntt_bo_closed_vs_fast(oracle, log2n):
    n = 1 << log2n
    q = oracle.find_primes(n, 1, 60)[0]
    psi = oracle.find_psi(q, n)
    r = random.Random(100 + log2n)
    a = _rand(r, n, q)
    f1 = oracle.ntt_fwd_bo(a, q, psi, closed=True)
    f2 = oracle.ntt_fwd_bo(a, q, psi)
    assert f1.tolist() == f2.tolist()
    assert oracle.ntt_inv_bo(f1, q, psi, closed=True).tolist() == a.tolist()
    assert oracle.ntt_inv_bo(f1, q, psi).tolist() == a.tolist()
    # the bo-order transform diagonalises the negacyclic product
    b = _rand(r, n, q)
    fb = oracle.ntt_fwd_bo(b, q, psi)
    prod = [(int(x) * int(y)) % q for x, y in zip(f2, fb)]
    assert oracle.ntt_inv_bo(prod, q, psi).tolist() == oracle.schoolbook(a, b, q).tolist()


# ------------------------------------------------------------- Barrett ------
@pytest.mark.parametrize("m", [4, 6, 8, 10])
def test_barrett_exhaustive_small_m(oracle, m):
    """Algorithms 2-4 return x mod q for every x < 2^{2m} and every q of bit
    length m (m <= 8) or a sample of them; Algorithms 3 and 4 never need more
    than one correction (Sec. II-B)."""
    qs = [q for q in range(1 << (m - 1), 1 << m) if q % 2 == 1]
    if m >= 10:
        qs = qs[:: max(1, len(qs) // 8)]
    xs = range(1 << (2 * m)) if m <= 8 else range(0, 1 << (2 * m), 7)
    for q in qs:
        for x in xs:
            for alg in (2, 3, 4):
                r, k = oracle.barrett(alg, x, q)
                assert r == x % q, (alg, q, x)
                if alg in (3, 4):
                    assert k <= 1


def test_barrett_alg4_random_60_62_bits(oracle):
    r = random.Random(11)
    for bits in (30, 60, 62):
        for q in oracle.find_primes(1 << 12, 3, bits):
            mu = oracle.barrett_alg4_mu(q)
            m = q.bit_length()
            assert mu == (1 << (2 * m + 1)) // q
            for _ in range(3000):
                a, b = r.randrange(q), r.randrange(q)
                res, k = oracle.barrett(4, a * b, q)
                assert res == (a * b) % q and k <= 1
            for a, b in [(0, 0), (1, q - 1), (q - 1, q - 1)]:
                assert oracle.barrett(4, a * b, q)[0] == (a * b) % q


@pytest.mark.parametrize("nthreads", [1, 3, 4])
def test_polymul_ntt_batch_limb_rotation(oracle, nthreads):
    """The batched CPU product (the timing harness of the CPU baseline) is the
    per-unit product with unit u on limb u mod L, for every thread split
    (7 units over 3 limbs: with 4 threads the chunks start at units 0, 2, 4,
    6, i.e. limb offsets 0, 2, 1, 0).  Each unit is also pinned to the
    schoolbook definition."""
    log2n, L, U = 6, 3, 7
    n = 1 << log2n
    qs = oracle.find_primes(n, L, 60)
    psis = [oracle.find_psi(q, n) for q in qs]
    rng = np.random.default_rng(2209)
    a = np.stack([rng.integers(0, qs[u % L], n, dtype=np.uint64) for u in range(U)])
    b = np.stack([rng.integers(0, qs[u % L], n, dtype=np.uint64) for u in range(U)])
    got = oracle.polymul_ntt_batch(a, b, qs, psis, nthreads=nthreads)
    for u in range(U):
        q = qs[u % L]
        assert np.array_equal(got[u], oracle.polymul_ntt(a[u], b[u], q, psis[u % L])), u
        assert np.array_equal(got[u], oracle.schoolbook(a[u], b[u], q)), u
