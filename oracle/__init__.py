"""CPU oracle for negacyclic polynomial multiplication (arxiv 2209.01290).

TEST INFRASTRUCTURE ONLY.  This package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` -- nothing else.  It shares no code with the GPU path
(``paper_2209_01290_gb300``) and never imports it.

The arithmetic lives in ``pm_oracle.c`` (plain C, ``unsigned __int128`` and
``%``); this module compiles it with gcc on first use and exposes numpy-level
wrappers.  See the C file for the paper passage each routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libpm_oracle.so")
_lock = threading.Lock()
_lib = None

_U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile pm_oracle.c into oracle/_build/libpm_oracle.so (gcc, -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        sig = {
            "or_mulmod": (u64, [u64, u64, u64]),
            "or_addmod": (u64, [u64, u64, u64]),
            "or_submod": (u64, [u64, u64, u64]),
            "or_powmod": (u64, [u64, u64, u64]),
            "or_invmod": (u64, [u64, u64]),
            "or_is_prime": (i32, [u64]),
            "or_find_primes": (i32, [u32, u32, u32, _U64P]),
            "or_find_psi": (u64, [u64, u32]),
            "or_bitrev": (u64, [u64, u32]),
            "or_bitlen": (u32, [u64]),
            "or_half": (u64, [u64, u64]),
            "or_schoolbook_negacyclic": (None, [u32, u64, _U64P, _U64P, _U64P]),
            "or_ntt_cyclic": (None, [u32, u64, u64, _U64P]),
            "or_polymul_ntt": (None, [u32, u64, u64, _U64P, _U64P, _U64P]),
            "or_polymul_ntt_batch": (None, [u32, u32, u32, _U64P, _U64P, _U64P, _U64P, _U64P]),
            "or_ntt_fwd_bo_closed": (None, [u32, u64, u64, _U64P, _U64P]),
            "or_ntt_inv_bo_closed": (None, [u32, u64, u64, _U64P, _U64P]),
            "or_ntt_fwd_bo": (None, [u32, u64, u64, _U64P, _U64P]),
            "or_ntt_inv_bo": (None, [u32, u64, u64, _U64P, _U64P]),
            "or_barrett_alg2": (u64, [u64, u64, u64, ctypes.POINTER(ctypes.c_int)]),
            "or_barrett_alg3": (u64, [u64, u64, u64, ctypes.POINTER(ctypes.c_int)]),
            "or_barrett_alg4": (u64, [u64, u64, u64, ctypes.POINTER(ctypes.c_int)]),
            "or_barrett_alg4_mu": (u64, [u64]),
            "or_polymul_eq2": (None, [u32, u64, u64, _U64P, _U64P, _U64P]),
            "or_polymul_alg8": (None, [u32, u64, u64, _U64P, _U64P, _U64P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(x: np.ndarray):
    assert x.dtype == np.uint64 and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(_U64P)


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


def _log2(n: int) -> int:
    if n < 1 or n & (n - 1):
        raise ValueError(f"N={n} is not a power of two")
    return n.bit_length() - 1


# ---------------------------------------------------------------- scalars
def mulmod(a: int, b: int, q: int) -> int:
    return int(_load().or_mulmod(a, b, q))


def powmod(a: int, e: int, q: int) -> int:
    return int(_load().or_powmod(a, e, q))


def invmod(a: int, q: int) -> int:
    return int(_load().or_invmod(a, q))


def half(x: int, q: int) -> int:
    """x/2 mod q by the even/odd rule of Sec. III-A (x in [0,q))."""
    return int(_load().or_half(x, q))


def is_prime(n: int) -> bool:
    return bool(_load().or_is_prime(n))


def bitrev(i: int, bits: int) -> int:
    return int(_load().or_bitrev(i, bits))


def bitlen(q: int) -> int:
    return int(_load().or_bitlen(q))


def find_primes(n: int, count: int, bits: int = 60) -> list[int]:
    """The `count` largest primes q < 2^bits with q = 1 mod 2N, descending."""
    out = np.zeros(max(count, 1), dtype=np.uint64)
    k = _load().or_find_primes(_log2(n), bits, count, _ptr(out))
    return [int(v) for v in out[:k]]


def find_psi(q: int, n: int) -> int:
    """First psi = x^((q-1)/2N), x = 2, 3, ..., with psi^N = -1 mod q."""
    return int(_load().or_find_psi(q, _log2(n)))


def barrett(alg: int, x: int, q: int) -> tuple[int, int]:
    """Algorithm 2, 3 or 4 on x < 2^128; returns (result, corrections taken)."""
    f = {2: "or_barrett_alg2", 3: "or_barrett_alg3", 4: "or_barrett_alg4"}[alg]
    k = ctypes.c_int(0)
    r = getattr(_load(), f)(x >> 64, x & ((1 << 64) - 1), q, ctypes.byref(k))
    return int(r), int(k.value)


def barrett_alg4_mu(q: int) -> int:
    return int(_load().or_barrett_alg4_mu(q))


# ---------------------------------------------------------------- vectors
def schoolbook(a, b, q: int) -> np.ndarray:
    """Negacyclic product by its definition, O(N^2)."""
    a, b = _u64(a), _u64(b)
    c = np.empty_like(a)
    _load().or_schoolbook_negacyclic(a.size, q, _ptr(a), _ptr(b), _ptr(c))
    return c


def ntt_cyclic(x, q: int, omega: int) -> np.ndarray:
    x = _u64(x).copy()
    _load().or_ntt_cyclic(_log2(x.size), q, omega, _ptr(x))
    return x


def polymul_ntt(a, b, q: int, psi: int) -> np.ndarray:
    """Negacyclic product via the psi-twisted textbook cyclic NTT."""
    a, b = _u64(a), _u64(b)
    c = np.empty_like(a)
    _load().or_polymul_ntt(_log2(a.size), q, psi, _ptr(a), _ptr(b), _ptr(c))
    return c


def polymul_ntt_batch(a, b, qs, psis, nthreads: int = 1) -> np.ndarray:
    """Batched scalar-NTT product over units [U][N]; unit u uses qs[u % L].

    With nthreads > 1 the units are split into contiguous chunks run on a
    thread pool (ctypes releases the GIL during each call)."""
    a, b = _u64(a), _u64(b)
    assert a.shape == b.shape and a.ndim == 2
    U, N = a.shape
    qs, psis = _u64(qs), _u64(psis)
    L = qs.size
    c = np.empty_like(a)
    lib = _load()
    log2n = _log2(N)

    def run(u0, u1):
        if u1 <= u0:
            return
        # keep the limb pattern: unit u -> limb u % L, so pass rotated tables
        rq = np.ascontiguousarray(np.roll(qs, -(u0 % L)))
        rp = np.ascontiguousarray(np.roll(psis, -(u0 % L)))
        lib.or_polymul_ntt_batch(log2n, u1 - u0, L, _ptr(rq), _ptr(rp),
                                 _ptr(a[u0:u1]), _ptr(b[u0:u1]), _ptr(c[u0:u1]))

    if nthreads <= 1 or U <= 1:
        run(0, U)
    else:
        import concurrent.futures as cf
        step = (U + nthreads - 1) // nthreads
        with cf.ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(lambda s: run(s, min(U, s + step)), range(0, U, step)))
    return c


def ntt_fwd_bo(a, q: int, psi: int, closed: bool = False) -> np.ndarray:
    """Forward negacyclic NTT, normal order in, bit-reversed order out."""
    a = _u64(a)
    out = np.empty_like(a)
    f = _load().or_ntt_fwd_bo_closed if closed else _load().or_ntt_fwd_bo
    f(_log2(a.size), q, psi, _ptr(a), _ptr(out))
    return out


def ntt_inv_bo(ahat, q: int, psi: int, closed: bool = False) -> np.ndarray:
    """Inverse of ntt_fwd_bo (bit-reversed in, normal order out, 1/N applied)."""
    ahat = _u64(ahat)
    out = np.empty_like(ahat)
    f = _load().or_ntt_inv_bo_closed if closed else _load().or_ntt_inv_bo
    f(_log2(ahat.size), q, psi, _ptr(ahat), _ptr(out))
    return out


def polymul_eq2(a, b, q: int, psi: int) -> np.ndarray:
    """Eq. 2 written out with Algorithms 6 and 7 (reading check)."""
    a, b = _u64(a), _u64(b)
    c = np.empty_like(a)
    _load().or_polymul_eq2(_log2(a.size), q, psi, _ptr(a), _ptr(b), _ptr(c))
    return c


def polymul_alg8(a, b, q: int, psi: int) -> np.ndarray:
    """Algorithm 8, fused polynomial multiplication (reading check), N >= 4."""
    a, b = _u64(a), _u64(b)
    c = np.empty_like(a)
    _load().or_polymul_alg8(_log2(a.size), q, psi, _ptr(a), _ptr(b), _ptr(c))
    return c


def polymul(a, b, q: int, psi: int) -> np.ndarray:
    """The oracle's answer for a negacyclic product: schoolbook up to N=2^10,
    the scalar textbook NTT above (the two are cross-pinned in the tests)."""
    a = _u64(a)
    if a.size <= 1024:
        return schoolbook(a, b, q)
    return polymul_ntt(a, b, q, psi)
