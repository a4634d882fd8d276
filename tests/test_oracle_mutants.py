"""Planted mistakes in the oracle must be caught by the pins (no GPU).

Each case copies oracle/pm_oracle.c, plants one plausible mistake (a dropped
term, a wrong sign, index or exponent, swapped operands), compiles the copy
into a temporary library, loads the oracle's Python wrappers against it and
runs a quick battery of the same kinds of pins as test_oracle_pins.py.  The
battery must reject every mutant, and accept the unmodified source.
"""
import importlib.util
import os
import random
import shutil
import tempfile

import numpy as np
import pytest

import oracle as _oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MUTANTS = {
    "schoolbook_wrap_sign": ("c[k] = (uint64_t)((pos + (u128)q - neg) % q);",
                             "c[k] = (uint64_t)((pos + neg) % q);"),
    "schoolbook_wrap_index": ("uint32_t j = k + n - i;", "uint32_t j = k + n - i - 1;"),
    "cyclic_swapped_sub": ("x[s + t + len / 2] = or_submod(u, v, q);",
                           "x[s + t + len / 2] = or_submod(v, u, q);"),
    "cyclic_dropped_twiddle_step": ("w = or_mulmod(w, wlen, q);", "(void)wlen;"),
    "polymul_dropped_ninv": ("c[i] = or_mulmod(or_mulmod(x[i], n_inv, q), pw, q);",
                             "c[i] = or_mulmod(x[i], pw, q);"),
    "polymul_untwist_sign": ("uint64_t psi_inv = or_invmod(psi, q);\n    uint64_t n_inv = or_invmod(n % q, q);\n    uint64_t pw = 1;\n    for (uint64_t i = 0; i < n; i++) {              /* Psi . a",
                             "uint64_t psi_inv = psi;\n    uint64_t n_inv = or_invmod(n % q, q);\n    uint64_t pw = 1;\n    for (uint64_t i = 0; i < n; i++) {              /* Psi . a"),
    "closed_fwd_exponent": ("uint64_t e = 2 * or_bitrev(j, log2n) + 1;",
                            "uint64_t e = 2 * or_bitrev(j, log2n);"),
    "fast_fwd_no_bitrev": ("for (uint64_t j = 0; j < n; j++) out[j] = x[or_bitrev(j, log2n)];",
                           "for (uint64_t j = 0; j < n; j++) out[j] = x[j];"),
    "alg4_shift": ("u128 quot = (c * mu) >> (m + 3);", "u128 quot = (c * mu) >> (m + 2);"),
    "alg6_sign": ("a[j + k] = or_submod(u, t, q);", "a[j + k] = or_addmod(u, t, q);"),
    "alg7_no_halving": ("a[j] = halve ? or_half(s, q) : s;", "a[j] = s;"),
    "half_wrong_constant": ("return (x & 1) ? (x >> 1) + (q + 1) / 2 : (x >> 1);",
                            "return (x & 1) ? (x >> 1) + (q - 1) / 2 : (x >> 1);"),
    "alg8_parity_sign": ("z[2 * i] = (i % 2 == 0) ? or_addmod(u, zz, q) : or_submod(u, zz, q);",
                         "z[2 * i] = (i % 2 == 1) ? or_addmod(u, zz, q) : or_submod(u, zz, q);"),
    "psi_accept_order_n": ("if (or_powmod(psi, n, q) == q - 1) return psi;",
                           "if (or_powmod(psi, 2 * n, q) == 1) return psi;"),
    "primes_wrong_step": ("cand -= step;", "cand -= 2;"),
    "mulmod_truncated": ("return (uint64_t)(((u128)a * (u128)b) % (u128)q);",
                         "return (uint64_t)(((uint64_t)(a * b)) % q);"),
}


def _load_variant(src_text, tmpdir):
    src = os.path.join(tmpdir, "pm_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    spec = importlib.util.spec_from_file_location(f"oracle_variant_{abs(hash(src_text))}",
                                                  _oracle.__file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = src
    mod._BUILD_DIR = os.path.join(tmpdir, "_build")
    mod._LIB_PATH = os.path.join(mod._BUILD_DIR, "libpm_oracle.so")
    mod._lib = None
    mod.build(force=True)
    return mod


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([list(map(int, p.split())) for p in line.split("|")])
    return out


def _numpy_negacyclic(a, b, q):
    n = len(a)
    p = np.convolve(np.array([int(x) for x in a], dtype=object),
                    np.array([int(x) for x in b], dtype=object))
    return [(int(p[k]) - (int(p[k + n]) if k + n < len(p) else 0)) % q for k in range(n)]


def _battery(o):
    """Returns the list of failed pin names (empty = all pins hold)."""
    failed = []

    def check(name, cond):
        if not cond:
            failed.append(name)

    try:
        for (n, q), a, b, c in _rows("negacyclic_small.txt"):
            check("golden_schoolbook", o.schoolbook(a, b, q).tolist() == c)
            psi = o.find_psi(q, n)
            check("golden_ntt_polymul", psi != 0 and o.polymul_ntt(a, b, q, psi).tolist() == c)
            check("golden_eq2", psi != 0 and o.polymul_eq2(a, b, q, psi).tolist() == c)
            if n >= 4:
                check("golden_alg8", psi != 0 and o.polymul_alg8(a, b, q, psi).tolist() == c)
        for (n, q, psi), a, ahat in _rows("ntt_bo_small.txt"):
            check("golden_psi", o.find_psi(q, n) == psi)
            check("golden_fwd_closed", o.ntt_fwd_bo(a, q, psi, closed=True).tolist() == ahat)
            check("golden_fwd_fast", o.ntt_fwd_bo(a, q, psi).tolist() == ahat)
            check("golden_inv_fast", o.ntt_inv_bo(ahat, q, psi).tolist() == a)
        r = random.Random(5)
        for n, q in [(16, 1152921504606830593), (32, 7681)]:
            a = [r.randrange(q) for _ in range(n)]
            b = [r.randrange(q) for _ in range(n)]
            want = _numpy_negacyclic(a, b, q)
            check("schoolbook_vs_numpy", o.schoolbook(a, b, q).tolist() == want)
            psi = o.find_psi(q, n)
            check("ntt_polymul_vs_numpy", psi != 0 and o.polymul_ntt(a, b, q, psi).tolist() == want)
            check("eq2_vs_numpy", psi != 0 and o.polymul_eq2(a, b, q, psi).tolist() == want)
            check("alg8_vs_numpy", psi != 0 and o.polymul_alg8(a, b, q, psi).tolist() == want)
        for _ in range(200):
            q = r.randrange(3, 1 << 62) | 1
            x, y = r.randrange(1 << 64), r.randrange(1 << 64)
            check("mulmod_vs_int", o.mulmod(x, y, q) == (x * y) % q)
        for q in (7681, 1152921504606830593):
            for _ in range(50):
                x = r.randrange(q)
                check("half_rule", (2 * o.half(x, q)) % q == x)
        for q in o.find_primes(1 << 12, 2, 60) + [994705409]:
            for _ in range(300):
                x, y = r.randrange(q), r.randrange(q)
                res, k = o.barrett(4, x * y, q)
                check("alg4_vs_int", res == (x * y) % q and k <= 1)
        qs = o.find_primes(1 << 16, 3, 60)
        check("primes_form", len(qs) == 3 and all((q - 1) % (1 << 17) == 0 for q in qs))
        import sympy
        check("primes_sympy", all(sympy.isprime(q) for q in qs))
        n = 1 << 12
        q = o.find_primes(n, 1, 60)[0]
        psi = o.find_psi(q, n)
        check("psi_order", psi != 0 and sympy.n_order(psi, q) == 2 * n)
    except Exception as e:  # a crash counts as a caught mutant
        failed.append(f"exception:{type(e).__name__}")
    return failed


@pytest.fixture(scope="module")
def clean_src():
    with open(_oracle._SRC) as f:
        return f.read()


def test_battery_accepts_clean_oracle(clean_src):
    d = tempfile.mkdtemp()
    try:
        assert _battery(_load_variant(clean_src, d)) == []
    finally:
        shutil.rmtree(d)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_battery_rejects_mutant(clean_src, name):
    old, new = MUTANTS[name]
    assert clean_src.count(old) == 1, f"mutation site for {name} not unique/absent"
    d = tempfile.mkdtemp()
    try:
        failed = _battery(_load_variant(clean_src.replace(old, new), d))
        assert failed, f"mutant {name} survived every pin"
    finally:
        shutil.rmtree(d)
