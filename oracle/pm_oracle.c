/*
 * pm_oracle.c -- plain, slow, obviously correct CPU oracle for negacyclic
 * polynomial multiplication in Z_q[X]/(X^N+1) (arxiv 2209.01290).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The GPU
 * product path never calls it and shares no code with it.
 *
 * Every routine is exact integer arithmetic on uint64 words with unsigned
 * __int128 intermediates and the C '%' operator as the reduction (the plain
 * definition of "x mod q", Sec. II-A).  No blocking, fusion, lazy ranges or
 * reordering beyond what each cited definition states.
 *
 * Contents (each function cites the passage it follows):
 *   or_mulmod / or_addmod / or_submod / or_powmod / or_invmod  -- Sec. II-A
 *   or_is_prime, or_find_primes, or_find_psi                   -- Sec. III-A setup
 *   or_bitrev                                                  -- Sec. III-A (br)
 *   or_schoolbook_negacyclic                                   -- Sec. III (naive O(N^2))
 *   or_ntt_cyclic                                              -- Sec. III-A (NTT_omega)
 *   or_polymul_ntt                                             -- Sec. III-A (psi-twist relation)
 *   or_ntt_fwd_bo_closed / or_ntt_inv_bo_closed                -- Eq. 1 convention, closed form
 *   or_ntt_fwd_bo / or_ntt_inv_bo                              -- same map via or_ntt_cyclic
 *   or_barrett_alg2 / or_barrett_alg3 / or_barrett_alg4        -- Algorithms 2, 3, 4
 *   or_polymul_eq2                                             -- Algorithms 6, 7 + Eq. 2 (reading check)
 *   or_polymul_alg8                                            -- Algorithm 8 (reading check)
 *
 * Pins: tests/test_oracle_*.py check these against hand-worked fixtures,
 * closed forms, library routines (sympy, numpy object convolution), brute
 * force and algebraic identities.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- basics */

/* (a*b) mod q by the definition of "mod" (Sec. II-A): full 128-bit product,
 * then the C remainder operator. */
uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % (u128)q);
}

/* (a+b) mod q, computed in 128 bits so no precondition on q is needed. */
uint64_t or_addmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)(a % q) + (u128)(b % q)) % (u128)q);
}

/* (a-b) mod q in [0,q). */
uint64_t or_submod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t x = a % q, y = b % q;
    return x >= y ? x - y : (uint64_t)((u128)x + q - y);
}

/* a^e mod q, square-and-multiply. */
uint64_t or_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q, b = a % q;
    while (e) {
        if (e & 1) r = or_mulmod(r, b, q);
        b = or_mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* a^{-1} mod q for prime q (Fermat). */
uint64_t or_invmod(uint64_t a, uint64_t q) { return or_powmod(a, q - 2, q); }

/* --------------------------------------------------------- setup (Sec. III-A) */

/* Deterministic Miller-Rabin for n < 2^64 with the first twelve prime bases
 * (a textbook result: these bases are exact for all 64-bit n). */
int or_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; r++) {
            x = or_mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/* The `count` largest primes q < 2^bits with 2N | q-1, in descending order
 * (the setup of Sec. III-A requires q prime with 2N dividing q-1).
 * Returns the number found (may be < count if the range is exhausted). */
int or_find_primes(uint32_t log2n, uint32_t bits, uint32_t count, uint64_t *out) {
    if (bits < 2 || bits > 63 || log2n + 1 >= bits) return 0;
    uint64_t step = (uint64_t)2 << log2n;            /* 2N */
    uint64_t top = (uint64_t)1 << bits;              /* exclusive bound */
    /* largest candidate of the form k*2N + 1 below 2^bits */
    uint64_t cand = ((top - 2) / step) * step + 1;
    uint32_t found = 0;
    uint64_t tried = 0;                 /* bounded: primes of this form are dense */
    while (found < count && cand > step && tried++ < ((uint64_t)1 << 24)) {
        if (or_is_prime(cand)) out[found++] = cand;
        cand -= step;
    }
    return (int)found;
}

/* A primitive 2N-th root of unity mod q (Sec. III-A, property 3).  The paper
 * does not say which one; the reading used throughout this project: for
 * x = 2, 3, 4, ... take psi = x^((q-1)/(2N)) and accept the first psi with
 * psi^N == q-1 (which certifies that its order is exactly 2N).
 * Returns 0 if none is found (q not = 1 mod 2N, or q not prime). */
uint64_t or_find_psi(uint64_t q, uint32_t log2n) {
    uint64_t two_n = (uint64_t)2 << log2n;
    if (q < 3 || (q - 1) % two_n != 0) return 0;
    uint64_t e = (q - 1) / two_n;
    uint64_t n = (uint64_t)1 << log2n;
    for (uint64_t x = 2; x < q && x < 4096; x++) {   /* bounded search */
        uint64_t psi = or_powmod(x, e, q);
        if (or_powmod(psi, n, q) == q - 1) return psi;
    }
    return 0;
}

/* br(i): reversal of the low `bits` bits of i (Sec. III, definition of br). */
uint64_t or_bitrev(uint64_t i, uint32_t bits) {
    uint64_t r = 0;
    for (uint32_t b = 0; b < bits; b++) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

/* ------------------------------------------------- polymul by definition */

/* Negacyclic convolution c = a*b in Z_q[X]/(X^N+1) (Sec. III: polynomial
 * multiplication is negacyclic convolution; the naive method is O(N^2)):
 *   c_k = sum_{i+j=k} a_i b_j  -  sum_{i+j=k+N} a_i b_j   (mod q).
 * The positive and negative parts are accumulated separately in 128 bits and
 * reduced with '%' before they can overflow (each product is < 2^126 for
 * q < 2^63, so at most one product is added between reductions). */
void or_schoolbook_negacyclic(uint32_t n, uint64_t q, const uint64_t *a,
                              const uint64_t *b, uint64_t *c) {
    for (uint32_t k = 0; k < n; k++) {
        u128 pos = 0, neg = 0;
        for (uint32_t i = 0; i < n; i++) {
            if (i <= k) {
                uint32_t j = k - i;               /* i + j = k      : +a_i b_j */
                pos = (pos + ((u128)(a[i] % q) * (b[j] % q)) % q) % q;
            } else {
                uint32_t j = k + n - i;           /* i + j = k + N  : -a_i b_j */
                neg = (neg + ((u128)(a[i] % q) * (b[j] % q)) % q) % q;
            }
        }
        c[k] = (uint64_t)((pos + (u128)q - neg) % q);
    }
}

/* ------------------------------------------------------ scalar textbook NTT */

/* In-place cyclic N-point NTT with respect to omega (Sec. III-A:
 * NTT_omega(x)_j = sum_i x_i omega^{ij}), computed by the textbook
 * iterative radix-2 decimation-in-time FFT: an explicit bit-reversal
 * permutation of the input, then log2 N doubling stages.  This is the
 * classical cyclic NTT; it shares no structure with the merged,
 * bit-reversed-table transforms of Algorithms 6 and 7. */
void or_ntt_cyclic(uint32_t log2n, uint64_t q, uint64_t omega, uint64_t *x) {
    uint64_t n = (uint64_t)1 << log2n;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t r = or_bitrev(i, log2n);
        if (r > i) { uint64_t t = x[i]; x[i] = x[r]; x[r] = t; }
    }
    for (uint64_t len = 2; len <= n; len <<= 1) {
        uint64_t wlen = or_powmod(omega, n / len, q);   /* primitive len-th root */
        for (uint64_t s = 0; s < n; s += len) {
            uint64_t w = 1;
            for (uint64_t t = 0; t < len / 2; t++) {
                uint64_t u = x[s + t];
                uint64_t v = or_mulmod(x[s + t + len / 2], w, q);
                x[s + t] = or_addmod(u, v, q);
                x[s + t + len / 2] = or_submod(u, v, q);
                w = or_mulmod(w, wlen, q);
            }
        }
    }
}

/* Negacyclic product through the psi-twisted cyclic NTT (Sec. III-A):
 *   a (*) b = Psi^{-1} . (1/N) NTT_{omega^{-1}}( NTT_omega(Psi . a) . NTT_omega(Psi . b) ),
 * with Psi[i] = psi^i, omega = psi^2.  N^{-1} is a modular inverse. */
void or_polymul_ntt(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *a,
                    const uint64_t *b, uint64_t *c) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t *x = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *y = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t omega = or_mulmod(psi, psi, q);
    uint64_t omega_inv = or_invmod(omega, q);
    uint64_t psi_inv = or_invmod(psi, q);
    uint64_t n_inv = or_invmod(n % q, q);
    uint64_t pw = 1;
    for (uint64_t i = 0; i < n; i++) {              /* Psi . a, Psi . b */
        x[i] = or_mulmod(a[i] % q, pw, q);
        y[i] = or_mulmod(b[i] % q, pw, q);
        pw = or_mulmod(pw, psi, q);
    }
    or_ntt_cyclic(log2n, q, omega, x);
    or_ntt_cyclic(log2n, q, omega, y);
    for (uint64_t i = 0; i < n; i++) x[i] = or_mulmod(x[i], y[i], q);   /* Hadamard */
    or_ntt_cyclic(log2n, q, omega_inv, x);
    pw = 1;
    for (uint64_t i = 0; i < n; i++) {              /* Psi^{-1} . (1/N) . */
        c[i] = or_mulmod(or_mulmod(x[i], n_inv, q), pw, q);
        pw = or_mulmod(pw, psi_inv, q);
    }
    free(x);
    free(y);
}

/* Batched form over independent (polynomial, limb) units, for timing the
 * oracle as the CPU baseline: unit u uses modulus q[u % nlimbs] and
 * psi[u % nlimbs]; operands are contiguous [nunits][N]. */
void or_polymul_ntt_batch(uint32_t log2n, uint32_t nunits, uint32_t nlimbs,
                          const uint64_t *q, const uint64_t *psi, const uint64_t *a,
                          const uint64_t *b, uint64_t *c) {
    uint64_t n = (uint64_t)1 << log2n;
    for (uint32_t u = 0; u < nunits; u++)
        or_polymul_ntt(log2n, q[u % nlimbs], psi[u % nlimbs], a + (uint64_t)u * n,
                       b + (uint64_t)u * n, c + (uint64_t)u * n);
}

/* ------------------------------------ forward/inverse NTT in the bo convention */

/* The merged CT NTT of Algorithm 6 maps normal order to bit-reversed order
 * (Eq. 1 and the no->bo discussion of Sec. III-A).  Its output is the
 * psi-twisted cyclic NTT read at bit-reversed positions, which written out is
 *   ahat[j] = sum_i a_i psi^{i (2 br(j) + 1)}   (mod q).
 * O(N^2) closed form, used at small N. */
void or_ntt_fwd_bo_closed(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *a,
                          uint64_t *out) {
    uint64_t n = (uint64_t)1 << log2n;
    for (uint64_t j = 0; j < n; j++) {
        uint64_t e = 2 * or_bitrev(j, log2n) + 1;      /* psi^{e} is the j-th root */
        uint64_t root = or_powmod(psi, e, q);
        u128 acc = 0;
        uint64_t pw = 1;
        for (uint64_t i = 0; i < n; i++) {
            acc = (acc + (u128)or_mulmod(a[i] % q, pw, q)) % q;
            pw = or_mulmod(pw, root, q);
        }
        out[j] = (uint64_t)acc;
    }
}

/* Inverse of the map above: a_i = N^{-1} sum_j ahat[j] psi^{-i (2 br(j) + 1)}. */
void or_ntt_inv_bo_closed(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *ahat,
                          uint64_t *out) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t psi_inv = or_invmod(psi, q);
    uint64_t n_inv = or_invmod(n % q, q);
    for (uint64_t i = 0; i < n; i++) {
        u128 acc = 0;
        for (uint64_t j = 0; j < n; j++) {
            uint64_t e = ((2 * or_bitrev(j, log2n) + 1) * i) % (2 * n);
            acc = (acc + (u128)or_mulmod(ahat[j] % q, or_powmod(psi_inv, e, q), q)) % q;
        }
        out[i] = or_mulmod((uint64_t)acc, n_inv, q);
    }
}

/* Same forward map at any N via the textbook cyclic NTT:
 * ahat[j] = NTT_omega(Psi . a)[br(j)]. */
void or_ntt_fwd_bo(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *a,
                   uint64_t *out) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t *x = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t pw = 1;
    for (uint64_t i = 0; i < n; i++) {
        x[i] = or_mulmod(a[i] % q, pw, q);
        pw = or_mulmod(pw, psi, q);
    }
    or_ntt_cyclic(log2n, q, or_mulmod(psi, psi, q), x);
    for (uint64_t j = 0; j < n; j++) out[j] = x[or_bitrev(j, log2n)];
    free(x);
}

/* Same inverse map at any N: a = Psi^{-1} . (1/N) NTT_{omega^{-1}}(x) with
 * x[br(j)] = ahat[j]. */
void or_ntt_inv_bo(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *ahat,
                   uint64_t *out) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t *x = (uint64_t *)malloc(n * sizeof(uint64_t));
    for (uint64_t j = 0; j < n; j++) x[or_bitrev(j, log2n)] = ahat[j] % q;
    uint64_t omega = or_mulmod(psi, psi, q);
    or_ntt_cyclic(log2n, q, or_invmod(omega, q), x);
    uint64_t psi_inv = or_invmod(psi, q);
    uint64_t n_inv = or_invmod(n % q, q);
    uint64_t pw = 1;
    for (uint64_t i = 0; i < n; i++) {
        out[i] = or_mulmod(or_mulmod(x[i], n_inv, q), pw, q);
        pw = or_mulmod(pw, psi_inv, q);
    }
    free(x);
}

/* ---------------------------------------------- Barrett variants (Sec. II-B) */

/* bit length len(q) = floor(log2 q) + 1 (Sec. II). */
uint32_t or_bitlen(uint64_t q) {
    uint32_t m = 0;
    while (q) { m++; q >>= 1; }
    return m;
}

/* Algorithm 2 (classical Barrett): m = len(q), mu = floor(2^{2m}/q),
 * c = x >> (m-1), quot = (c*mu) >> (m+1), rem = x - quot*q, then up to two
 * conditional subtractions.  x is given as (xhi, xlo).  *ncorr receives the
 * number of subtractions taken.  All intermediates in 128 bits (x < 2^{2m},
 * m <= 62). */
uint64_t or_barrett_alg2(uint64_t xhi, uint64_t xlo, uint64_t q, int *ncorr) {
    uint32_t m = or_bitlen(q);
    u128 x = ((u128)xhi << 64) | xlo;
    u128 mu = (((u128)1) << (2 * m)) / q;
    u128 c = x >> (m - 1);
    u128 quot = (c * mu) >> (m + 1);       /* c < 2^{m+1}, mu < 2^{m+1}: < 2^{2m+2} */
    u128 rem = x - quot * q;
    int k = 0;
    if (rem >= q) { rem -= q; k++; }
    if (rem >= q) { rem -= q; k++; }
    if (ncorr) *ncorr = k;
    return (uint64_t)rem;
}

/* Algorithm 3 (Dhem-Quisquater, alpha = N+3, beta = -2): mu = floor(2^{2m+3}/q),
 * c = x >> (m-2), quot = (c*mu) >> (m+5), one conditional subtraction.
 * Returns the result of those steps; *ncorr counts subtractions (the second
 * one, if it were ever needed, is counted but the paper's algorithm stops
 * after one -- the caller can check rem < q). */
uint64_t or_barrett_alg3(uint64_t xhi, uint64_t xlo, uint64_t q, int *ncorr) {
    uint32_t m = or_bitlen(q);
    u128 x = ((u128)xhi << 64) | xlo;
    u128 mu = (((u128)1) << (2 * m + 3)) / q;
    u128 c = x >> (m - 2);
    u128 quot = (c * mu) >> (m + 5);
    u128 rem = x - quot * q;
    int k = 0;
    if (rem >= q) { rem -= q; k++; }
    if (ncorr) *ncorr = k;
    return (uint64_t)rem;
}

/* Algorithm 4 (the paper's proposal; Dhem-Quisquater alpha = N+1, beta = -2):
 * REQUIRE m = len(q) <= beta-2, 0 <= x < 2^{2m}, mu = floor(2^{2m+1}/q);
 * c = x >> (m-2); quot = (c*mu) >> (m+3); rem = x - quot*q; one conditional
 * subtraction.  Same conventions as above. */
uint64_t or_barrett_alg4(uint64_t xhi, uint64_t xlo, uint64_t q, int *ncorr) {
    uint32_t m = or_bitlen(q);
    u128 x = ((u128)xhi << 64) | xlo;
    u128 mu = (((u128)1) << (2 * m + 1)) / q;
    u128 c = x >> (m - 2);
    /* c < 2^{m+2}, mu < 2^{m+2}: the product can exceed 2^128 only if
     * 2m+4 > 128, i.e. m > 62; callers respect m <= 62. */
    u128 quot = (c * mu) >> (m + 3);
    u128 rem = x - quot * q;
    int k = 0;
    if (rem >= q) { rem -= q; k++; }
    if (ncorr) *ncorr = k;
    return (uint64_t)rem;
}

/* The Barrett constant of Algorithm 4, floor(2^{2m+1}/q), m = len(q) <= 62. */
uint64_t or_barrett_alg4_mu(uint64_t q) {
    uint32_t m = or_bitlen(q);
    return (uint64_t)((((u128)1) << (2 * m + 1)) / q);
}

/* ---------------------------- reading checks: Eq. 2 and Algorithm 8 as written */

/* Psi_br[i] = w^{br(i)} over log2 N bits, for w = psi or psi^{-1}
 * (the permuted twiddle table required by Algorithms 6 and 7). */
static void or_table_br(uint32_t log2n, uint64_t q, uint64_t w, uint64_t *t) {
    uint64_t n = (uint64_t)1 << log2n;
    for (uint64_t i = 0; i < n; i++) t[i] = or_powmod(w, or_bitrev(i, log2n), q);
}

/* Algorithm 6 (merged CT NTT, no->bo), exactly as stated, every product and
 * sum reduced with '%'. */
static void or_alg6(uint32_t log2n, uint64_t q, const uint64_t *psi_br, uint64_t *a) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t m = 1, k = n / 2;
    while (m < n) {
        for (uint64_t i = 0; i < m; i++) {
            uint64_t j_first = 2 * i * k, j_last = j_first + k - 1;
            uint64_t xi = psi_br[m + i];
            for (uint64_t j = j_first; j <= j_last; j++) {
                uint64_t t = or_mulmod(xi, a[j + k], q);
                uint64_t u = a[j];
                a[j] = or_addmod(u, t, q);
                a[j + k] = or_submod(u, t, q);
            }
        }
        m *= 2;
        k /= 2;
    }
}

/* x/2 mod q by the case split of Sec. III-A (Zhang et al.): x/2 if x is even,
 * floor(x/2) + (q+1)/2 if x is odd; x in [0,q). */
uint64_t or_half(uint64_t x, uint64_t q) {
    return (x & 1) ? (x >> 1) + (q + 1) / 2 : (x >> 1);
}

/* Algorithm 7 (merged GS NTT, bo->no) with the table built from psi^{-1}
 * (Eq. 1 calls it with psi^{-1}), and, when `halve` is set, each butterfly
 * output multiplied by 1/2 (the 1/2-scaled variant used in Eq. 2).
 * `stop_m` ends the stage loop while m >= stop_m (1 = full transform,
 * 2 = truncated GS of Sec. III-B, which omits the first stage). */
static void or_alg7(uint32_t log2n, uint64_t q, const uint64_t *psiinv_br, uint64_t *a,
                    int halve, uint64_t start_m) {
    uint64_t m = start_m, k = ((uint64_t)1 << log2n) / (2 * start_m);
    while (m >= 1) {
        for (uint64_t i = 0; i < m; i++) {
            uint64_t j_first = 2 * i * k, j_last = j_first + k - 1;
            uint64_t xi = psiinv_br[m + i];
            for (uint64_t j = j_first; j <= j_last; j++) {
                uint64_t u = a[j], v = a[j + k];
                uint64_t s = or_addmod(u, v, q);
                uint64_t d = or_mulmod(xi, or_submod(u, v, q), q);
                a[j] = halve ? or_half(s, q) : s;
                a[j + k] = halve ? or_half(d, q) : d;
            }
        }
        m /= 2;
        k *= 2;
    }
}

/* Eq. 2: a (*) b = NTT^{GS,psi^{-1}}_{bo->no,1/2}( NTT^{CT,psi}(a) . NTT^{CT,psi}(b) ),
 * written out with Algorithms 6 and 7 as stated.  This is not the primary
 * oracle (the schoolbook is); it pins the readings of the inverse table and
 * of the 1/2 scaling against the schoolbook. */
void or_polymul_eq2(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *a,
                    const uint64_t *b, uint64_t *c) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t *tf = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *ti = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *x = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *y = (uint64_t *)malloc(n * sizeof(uint64_t));
    or_table_br(log2n, q, psi, tf);
    or_table_br(log2n, q, or_invmod(psi, q), ti);
    for (uint64_t i = 0; i < n; i++) { x[i] = a[i] % q; y[i] = b[i] % q; }
    or_alg6(log2n, q, tf, x);
    or_alg6(log2n, q, tf, y);
    for (uint64_t i = 0; i < n; i++) x[i] = or_mulmod(x[i], y[i], q);
    or_alg7(log2n, q, ti, x, 1, n / 2);
    memcpy(c, x, n * sizeof(uint64_t));
    free(tf); free(ti); free(x); free(y);
}

/* Algorithm 8 (fused polynomial multiplication), as stated: truncated CT
 * (final stage omitted) on a and b, the Karatsuba pair product with
 * Psi_br[N/4 + floor(i/2)] and a sign set by the parity of i, then the
 * truncated GS (first stage omitted) with the 1/2 scaling kept in its
 * remaining stages.  Requires N >= 4.  Reading check for the fused variant. */
void or_polymul_alg8(uint32_t log2n, uint64_t q, uint64_t psi, const uint64_t *a,
                     const uint64_t *b, uint64_t *c) {
    uint64_t n = (uint64_t)1 << log2n;
    uint64_t *tf = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *ti = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *x = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *y = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *z = (uint64_t *)malloc(n * sizeof(uint64_t));
    or_table_br(log2n, q, psi, tf);
    or_table_br(log2n, q, or_invmod(psi, q), ti);
    for (uint64_t i = 0; i < n; i++) { x[i] = a[i] % q; y[i] = b[i] % q; }
    /* truncated CT: Algorithm 6 with "while m < N/2" */
    for (int pass = 0; pass < 2; pass++) {
        uint64_t *v = pass ? y : x;
        uint64_t m = 1, k = n / 2;
        while (m < n / 2) {
            for (uint64_t i = 0; i < m; i++) {
                uint64_t xi = tf[m + i];
                for (uint64_t j = 2 * i * k; j < 2 * i * k + k; j++) {
                    uint64_t t = or_mulmod(xi, v[j + k], q), u = v[j];
                    v[j] = or_addmod(u, t, q);
                    v[j + k] = or_submod(u, t, q);
                }
            }
            m *= 2;
            k /= 2;
        }
    }
    for (uint64_t i = 0; i < n / 2; i++) {
        uint64_t u = or_mulmod(x[2 * i], y[2 * i], q);
        uint64_t v = or_mulmod(x[2 * i + 1], y[2 * i + 1], q);
        uint64_t w = or_mulmod(or_addmod(x[2 * i], x[2 * i + 1], q),
                               or_addmod(y[2 * i], y[2 * i + 1], q), q);
        uint64_t yy = or_submod(w, u, q);
        z[2 * i + 1] = or_submod(yy, v, q);
        uint64_t zz = or_mulmod(v, tf[n / 4 + i / 2], q);
        z[2 * i] = (i % 2 == 0) ? or_addmod(u, zz, q) : or_submod(u, zz, q);
    }
    /* truncated GS: Algorithm 7 (1/2-scaled) with its first stage (m = N/2,
     * k = 1) omitted, i.e. starting at m = N/4, k = 2 and running down to m = 1.
     * The text's "while m > 1" would drop the last stage instead; the prose
     * ("first stage omitted") and Expr. 3 fix this reading. */
    if (n >= 4) or_alg7(log2n, q, ti, z, 1, n / 4);
    memcpy(c, z, n * sizeof(uint64_t));
    free(tf); free(ti); free(x); free(y); free(z);
}
