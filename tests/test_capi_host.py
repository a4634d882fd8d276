"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/*.h, and its host-side setup (parameter search, argument
validation) behaves as documented.  The parameter search is compared with the
oracle's independently written search and with sympy."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2209_01290_gb300 import capi
    return capi.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ["pm_plan_create", "pm_plan_destroy", "pm_ntt_fwd", "pm_ntt_inv",
                 "pm_pointwise", "pm_polymul", "pm_find_params", "pm_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2209_01290_gb300 import capi
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared function
    assert _declared() <= set(capi.SIGNATURES)


def test_version(lib):
    from paper_2209_01290_gb300 import capi
    assert re.match(r"\d+\.\d+\.\d+", capi.pm_version())


@pytest.mark.parametrize("log2n", [1, 4, 12, 13, 14, 15, 16, 17])
def test_find_params_matches_oracle(oracle, log2n):
    from paper_2209_01290_gb300 import capi
    L = 4 if log2n < 17 else 48
    qs, psis = capi.pm_find_params(log2n, L, 60)
    assert qs == oracle.find_primes(1 << log2n, L, 60)
    for q, psi in zip(qs, psis):
        assert psi == oracle.find_psi(q, 1 << log2n)


def test_find_params_config_primes(oracle):
    """The 32 limbs of the batched N=2^16 workload, checked with sympy."""
    import sympy
    from paper_2209_01290_gb300 import capi
    qs, psis = capi.pm_find_params(16, 32, 60)
    assert len(set(qs)) == 32 and all(q < (1 << 60) for q in qs)
    for q, psi in zip(qs, psis):
        assert (q - 1) % (1 << 17) == 0 and sympy.isprime(q)
        assert pow(psi, 1 << 16, q) == q - 1
    assert qs[0] == 0xffffffffffc0001
    # 62- and 30-bit variants
    q62, _ = capi.pm_find_params(16, 2, 62)
    assert q62 == oracle.find_primes(1 << 16, 2, 62)
    q30, _ = capi.pm_find_params(12, 2, 30)
    assert q30 == oracle.find_primes(1 << 12, 2, 30)


def test_find_params_errors():
    from paper_2209_01290_gb300 import capi
    with pytest.raises(capi.PMError) as e:
        capi.pm_find_params(18, 1, 60)
    assert e.value.status == -2
    with pytest.raises(capi.PMError) as e:
        capi.pm_find_params(16, 1, 63)
    assert e.value.status == -3
    with pytest.raises(capi.PMError) as e:
        capi.pm_find_params(16, 0, 60)
    assert e.value.status == -1
    # too few primes of the form below 2^20 for N = 2^17
    with pytest.raises(capi.PMError) as e:
        capi.pm_find_params(17, 50, 20)
    assert e.value.status == -3


def _create(lib, log2n, qs, psis=None, device=0):
    L = len(qs)
    q = (ctypes.c_uint64 * L)(*qs)
    p = (ctypes.c_uint64 * L)(*psis) if psis is not None else None
    out = ctypes.c_void_p()
    st = lib.pm_plan_create(ctypes.byref(out), log2n, L, q, p, device)
    return st, out


def test_plan_create_validation_before_device(lib):
    """Parameter errors are reported before any device work."""
    q16 = 0xffffffffffc0001
    # N out of range
    assert _create(lib, 18, [q16])[0] == -2
    assert _create(lib, 0, [q16])[0] == -2
    # q not = 1 mod 2N
    assert _create(lib, 16, [q16 + 2])[0] == -3
    # q composite but of the right form
    assert _create(lib, 4, [17 * 97])[0] == -3
    # q >= 2^62 (Algorithm 4 needs len(q) <= 62); 0xFFFFFFFF00000001 also fails
    assert _create(lib, 4, [0xFFFFFFFF00000001])[0] == -3
    # psi of order N (psi^2), not 2N
    import oracle as o
    psi = o.find_psi(q16, 1 << 16)
    assert _create(lib, 16, [q16], [pow(psi, 2, q16)])[0] == -4
    assert _create(lib, 16, [q16], [0])[0] == -4
    assert "psi" in lib.pm_last_error().decode()
    # null q / out
    assert lib.pm_plan_create(None, 4, 1, None, None, 0) == -1


def test_null_plan_calls(lib):
    assert lib.pm_polymul(None, None, None, None, 1, None) == -1
    assert lib.pm_ntt_fwd(None, None, 1, None) == -1
    assert lib.pm_plan_destroy(None) == 0
    buf = ctypes.create_string_buffer(64)
    lib.pm_ntt_inv(None, None, 1, None)
    assert lib.pm_last_error_string(buf, 64) == 0 and b"NULL" in buf.value
