"""ctypes binding of the C ABI in include/pm.h (argument marshalling only).

Every function here has the name of the C entry point it calls and passes
plain integers/pointers through; all arithmetic runs in libpm_gb300.so.
Loading fails loudly if the library has not been built or cannot be loaded:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PM_OK = 0
STATUS_NAMES = {
    0: "PM_OK", -1: "PM_ERR_ARG", -2: "PM_ERR_N", -3: "PM_ERR_Q", -4: "PM_ERR_PSI",
    -5: "PM_ERR_CUDA", -6: "PM_ERR_OOM", -7: "PM_ERR_TIMEOUT", -8: "PM_ERR_BUDGET",
    -9: "PM_ERR_UNSUPPORTED", -10: "PM_ERR_RANGE",
}

# exported symbol -> (restype, argtypes)
_u32, _u64, _i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_vp, _sz = ctypes.c_void_p, ctypes.c_size_t
_pu64, _pu32 = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
SIGNATURES = {
    "pm_find_params": (_i32, [_u32, _u32, _u32, _pu64, _pu64]),
    "pm_plan_create": (_i32, [ctypes.POINTER(_vp), _u32, _u32, _pu64, _pu64, _i32]),
    "pm_plan_create_ex": (_i32, [ctypes.POINTER(_vp), _u32, _u32, _pu64, _pu64, _i32, _u32]),
    "pm_plan_flags": (_i32, [_vp, _pu32]),
    "pm_plan_destroy": (_i32, [_vp]),
    "pm_plan_reserve": (_i32, [_vp, _u32, _vp]),
    "pm_plan_info": (_i32, [_vp, _pu32, _pu32, _pu64, _pu64]),
    "pm_ntt_fwd": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_ntt_inv": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_pointwise": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp]),
    "pm_polymul": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp]),
    "pm_polymul_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp]),
    "pm_polymul_noalloc": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp]),
    "pm_check_reduced": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_ntt_fwd32": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_ntt_inv32": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_pointwise32": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp]),
    "pm_polymul32": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp]),
    "pm_check_reduced32": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_plan_sync": (_i32, [_vp, _vp]),
    "pm_plan_tune": (_i32, [_vp, ctypes.c_void_p]),
    "pm_plan_inject_fault": (_i32, [_vp, _i32]),
    "pm_plan_autotune": (_i32, [_vp, _u32, _vp, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "pm_plan_get_tuning": (_i32, [_vp, ctypes.c_void_p]),
    "pm_plan_resolve_tuning": (_i32, [_vp, _u32, ctypes.c_void_p]),
    "pm_plan_set_phase_events": (_i32, [_vp, ctypes.POINTER(_vp), _i32]),
    "pm_last_error": (ctypes.c_char_p, []),
    "pm_last_error_string": (_i32, [ctypes.c_char_p, _sz]),
    "pm_version": (ctypes.c_char_p, []),
    "pm_measure_peaks": (_i32, [_i32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]),
    "pm_graph_create_polymul": (_i32, [ctypes.POINTER(_vp), _vp, _vp, _vp, _vp, _u32]),
    "pm_graph_launch": (_i32, [_vp, _vp]),
    "pm_graph_destroy": (_i32, [_vp]),
    "pm_reduction_rates": (_i32, [_i32, _u64, ctypes.POINTER(ctypes.c_double)]),
    "pm_reduction_apply": (_i32, [_i32, _u64, _vp, _vp, _vp, _u64, _vp]),
    "pm_server_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.c_void_p]),
    "pm_server_destroy": (_i32, [_vp]),
    "pm_server_submit": (_i32, [_vp, _vp, _vp, _vp, _u32, ctypes.POINTER(ctypes.c_uint64)]),
    "pm_server_wait": (_i32, [_vp, _u64, _u32, ctypes.POINTER(ctypes.c_void_p),
                              ctypes.POINTER(ctypes.c_double)]),
    "pm_server_release": (_i32, [_vp, _u64]),
    "pm_server_get_stats": (_i32, [_vp, ctypes.c_void_p]),
    "pm_queue_create": (_i32, [ctypes.POINTER(_vp), _i32]),
    "pm_queue_destroy": (_i32, [_vp]),
    "pm_queue_reserve": (_i32, [_vp, _u64, _u64]),
    "pm_polymul_uneven": (_i32, [_vp, _vp, _u32, _vp]),
    "pm_queue_sync": (_i32, [_vp, _vp]),
    "pm_queue_set_mode": (_i32, [_vp, _i32]),
}

_lib = None
_lock = threading.Lock()


class PMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpm_gb300.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libpm_gb300.so not built ({_build.LIB}); run "
                              "python -m paper_2209_01290_gb300.build")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != PM_OK:
        msg = load().pm_last_error().decode(errors="replace")
        raise PMError(status, where, msg)


def _call(name, *args):
    st = getattr(load(), name)(*args)
    check(st, name)


def pm_find_params(log2n: int, nlimbs: int, qbits: int = 60):
    q = (ctypes.c_uint64 * nlimbs)()
    psi = (ctypes.c_uint64 * nlimbs)()
    _call("pm_find_params", log2n, nlimbs, qbits, q, psi)
    return list(q), list(psi)


PM_PLAN_HALVING = 1
PM_PLAN_FUSED = 2
PM_PLAN_WORD32 = 4


def pm_plan_create(log2n: int, qs, psis=None, device: int = 0) -> int:
    return pm_plan_create_ex(log2n, qs, psis, device, 0)


def pm_plan_create_ex(log2n: int, qs, psis=None, device: int = 0, flags: int = 0) -> int:
    L = len(qs)
    q = (ctypes.c_uint64 * L)(*[int(x) for x in qs])
    p = (ctypes.c_uint64 * L)(*[int(x) for x in psis]) if psis is not None else None
    out = ctypes.c_void_p()
    _call("pm_plan_create_ex", ctypes.byref(out), log2n, L, q, p, device, flags)
    return out.value


def pm_plan_flags(plan: int) -> int:
    f = ctypes.c_uint32()
    _call("pm_plan_flags", plan, ctypes.byref(f))
    return f.value


def pm_plan_destroy(plan: int) -> None:
    _call("pm_plan_destroy", plan)


def pm_plan_reserve(plan: int, npoly: int, stream: int = 0) -> None:
    _call("pm_plan_reserve", plan, npoly, stream)


def pm_plan_info(plan: int):
    log2n, nl = ctypes.c_uint32(), ctypes.c_uint32()
    _call("pm_plan_info", plan, ctypes.byref(log2n), ctypes.byref(nl), None, None)
    L = nl.value
    q = (ctypes.c_uint64 * L)()
    psi = (ctypes.c_uint64 * L)()
    _call("pm_plan_info", plan, None, None, q, psi)
    return log2n.value, L, list(q), list(psi)


def pm_ntt_fwd(plan: int, d_x: int, npoly: int, stream: int = 0) -> None:
    _call("pm_ntt_fwd", plan, d_x, npoly, stream)


def pm_ntt_inv(plan: int, d_x: int, npoly: int, stream: int = 0) -> None:
    _call("pm_ntt_inv", plan, d_x, npoly, stream)


def pm_pointwise(plan: int, d_a: int, d_b: int, d_c: int, npoly: int, stream: int = 0) -> None:
    _call("pm_pointwise", plan, d_a, d_b, d_c, npoly, stream)


def pm_polymul(plan: int, d_a: int, d_b: int, d_c: int, npoly: int, stream: int = 0) -> None:
    _call("pm_polymul", plan, d_a, d_b, d_c, npoly, stream)


def pm_polymul_noalloc(plan: int, d_a: int, d_b: int, d_c: int, npoly: int,
                       stream: int = 0) -> None:
    """Allocation-free product (fixed 16 MiB library scratch, see pm.h)."""
    _call("pm_polymul_noalloc", plan, d_a, d_b, d_c, npoly, stream)


def pm_polymul_host(plan: int, h_a: int, h_b: int, h_c: int, d_a: int, d_b: int, d_c: int,
                    npoly: int, stream: int = 0) -> None:
    _call("pm_polymul_host", plan, h_a, h_b, h_c, d_a, d_b, d_c, npoly, stream)


def pm_check_reduced(plan: int, d_x: int, npoly: int, stream: int = 0) -> bool:
    st = load().pm_check_reduced(plan, d_x, npoly, stream)
    if st == -10:
        return False
    check(st, "pm_check_reduced")
    return True


# 32-bit words (plans with PM_PLAN_WORD32): the same calls on uint32 arrays.
def pm_ntt_fwd32(plan: int, d_x: int, npoly: int, stream: int = 0) -> None:
    _call("pm_ntt_fwd32", plan, d_x, npoly, stream)


def pm_ntt_inv32(plan: int, d_x: int, npoly: int, stream: int = 0) -> None:
    _call("pm_ntt_inv32", plan, d_x, npoly, stream)


def pm_pointwise32(plan: int, d_a: int, d_b: int, d_c: int, npoly: int, stream: int = 0) -> None:
    _call("pm_pointwise32", plan, d_a, d_b, d_c, npoly, stream)


def pm_polymul32(plan: int, d_a: int, d_b: int, d_c: int, npoly: int, stream: int = 0) -> None:
    _call("pm_polymul32", plan, d_a, d_b, d_c, npoly, stream)


def pm_check_reduced32(plan: int, d_x: int, npoly: int, stream: int = 0) -> bool:
    st = load().pm_check_reduced32(plan, d_x, npoly, stream)
    if st == -10:
        return False
    check(st, "pm_check_reduced32")
    return True


def pm_plan_set_phase_events(plan: int, events) -> None:
    """events: list of cudaEvent_t handles (ints), at most 4; [] turns it off."""
    arr = (ctypes.c_void_p * max(1, len(events)))(*[int(e) for e in events])
    _call("pm_plan_set_phase_events", plan, arr, len(events))


PM_VARIANT_SPLIT = 0
PM_VARIANT_PERSISTENT = 1


class PmTuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("ctas_per_sm", ctypes.c_uint32),
                ("lag_fwd", ctypes.c_uint32), ("lag_inv", ctypes.c_uint32),
                ("row_ops", ctypes.c_uint32)]

    def as_dict(self):
        return {"variant": "persistent" if self.variant == PM_VARIANT_PERSISTENT else "split",
                "ctas_per_sm": self.ctas_per_sm, "lag_fwd": self.lag_fwd,
                "lag_inv": self.lag_inv, "row_ops": self.row_ops}


def pm_plan_tune(plan: int, variant: int, ctas_per_sm: int = 4, lag_fwd: int = 8,
                 lag_inv: int = 64, row_ops: int = 0) -> None:
    t = PmTuning(variant, ctas_per_sm, lag_fwd, lag_inv, row_ops)
    _call("pm_plan_tune", plan, ctypes.byref(t))


def pm_plan_autotune(plan: int, npoly: int, stream: int = 0):
    """Time the launch choices for this batch size; returns (PmTuning, ms)."""
    t, ms = PmTuning(), ctypes.c_float()
    _call("pm_plan_autotune", plan, npoly, stream, ctypes.byref(t), ctypes.byref(ms))
    return t, ms.value


PM_FAULT_WITHHOLD_SIGNAL = 1
PM_FAULT_SHORT_TWIDDLES = 2


def pm_plan_inject_fault(plan: int, kind: int) -> None:
    _call("pm_plan_inject_fault", plan, kind)


def pm_plan_get_tuning(plan: int) -> PmTuning:
    t = PmTuning()
    _call("pm_plan_get_tuning", plan, ctypes.byref(t))
    return t


def pm_plan_resolve_tuning(plan: int, npoly: int) -> PmTuning:
    """The launch choice for a batch of npoly polynomials (row_ops resolved)."""
    t = PmTuning()
    _call("pm_plan_resolve_tuning", plan, npoly, ctypes.byref(t))
    return t


def pm_plan_sync(plan: int, stream: int = 0) -> None:
    _call("pm_plan_sync", plan, stream)


def pm_last_error() -> str:
    return load().pm_last_error().decode(errors="replace")


def pm_measure_peaks(device: int = 0):
    """(Shoup mulmods/s, 32-bit IMAD/s) measured on `device`."""
    m, i = ctypes.c_double(), ctypes.c_double()
    st = load().pm_measure_peaks(device, ctypes.byref(m), ctypes.byref(i))
    check(st, "pm_measure_peaks")
    return m.value, i.value


def pm_graph_create_polymul(plan: int, d_a: int, d_b: int, d_c: int, npoly: int) -> int:
    out = ctypes.c_void_p()
    _call("pm_graph_create_polymul", ctypes.byref(out), plan, d_a, d_b, d_c, npoly)
    return out.value


def pm_graph_launch(g: int, stream: int = 0) -> None:
    _call("pm_graph_launch", g, stream)


def pm_graph_destroy(g: int) -> None:
    _call("pm_graph_destroy", g)


class PmJob(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("npoly", ctypes.c_uint32)]


PM_UNEVEN_AUTO, PM_UNEVEN_PERSISTENT, PM_UNEVEN_GROUPED = 0, 1, 2


def pm_queue_set_mode(q: int, mode: int) -> None:
    _call("pm_queue_set_mode", q, mode)


def pm_queue_create(device: int = 0) -> int:
    out = ctypes.c_void_p()
    _call("pm_queue_create", ctypes.byref(out), device)
    return out.value


def pm_queue_destroy(q: int) -> None:
    _call("pm_queue_destroy", q)


def pm_queue_reserve(q: int, units: int, scratch_words: int) -> None:
    _call("pm_queue_reserve", q, units, scratch_words)


def pm_polymul_uneven(q: int, jobs, stream: int = 0) -> None:
    """jobs: sequence of (plan handle, d_a, d_b, d_c, npoly)."""
    arr = (PmJob * max(1, len(jobs)))(*[PmJob(*j) for j in jobs])
    _call("pm_polymul_uneven", q, arr, len(jobs), stream)


def pm_queue_sync(q: int, stream: int = 0) -> None:
    _call("pm_queue_sync", q, stream)


REDUCTIONS = ["builtin %", "alg2 (classical Barrett)", "alg3 (Dhem-Quisquater)",
              "alg4 (paper's Barrett)", "shoup (constant operand)", "montgomery"]


def pm_reduction_rates(device: int, q: int) -> dict:
    r = (ctypes.c_double * 6)()
    _call("pm_reduction_rates", device, q, r)
    return {name: r[i] for i, name in enumerate(REDUCTIONS)}


def pm_reduction_apply(variant: int, q: int, d_a: int, d_b: int, d_c: int, n: int,
                       stream: int = 0) -> None:
    _call("pm_reduction_apply", variant, q, d_a, d_b, d_c, n, stream)


class PmServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("min_batch_rows", ctypes.c_uint64)]


class PmServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("submitted", "completed", "batches", "batched_requests", "max_batch",
                 "arena_peak_bytes", "arena_used_bytes", "max_inflight", "max_device_overlap")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


def pm_server_create(device: int, budget_bytes: int, max_batch: int = 0, max_inflight: int = 2,
                     min_batch_rows: int = 0) -> int:
    cfg = PmServerConfig(budget_bytes, max_batch, max_inflight, min_batch_rows)
    out = ctypes.c_void_p()
    _call("pm_server_create", ctypes.byref(out), device, ctypes.byref(cfg))
    return out.value


def pm_server_destroy(s: int) -> None:
    _call("pm_server_destroy", s)


def pm_server_submit(s: int, plan: int, d_a: int, d_b: int, npoly: int) -> int:
    rid = ctypes.c_uint64()
    _call("pm_server_submit", s, plan, d_a, d_b, npoly, ctypes.byref(rid))
    return rid.value


def pm_server_wait(s: int, rid: int, timeout_ms: int = 60000):
    """(device pointer of the output, latency in microseconds)."""
    ptr, lat = ctypes.c_void_p(), ctypes.c_double()
    _call("pm_server_wait", s, rid, timeout_ms, ctypes.byref(ptr), ctypes.byref(lat))
    return ptr.value, lat.value


def pm_server_release(s: int, rid: int) -> None:
    _call("pm_server_release", s, rid)


def pm_server_get_stats(s: int) -> dict:
    st = PmServerStats()
    _call("pm_server_get_stats", s, ctypes.byref(st))
    return st.as_dict()


def pm_version() -> str:
    return load().pm_version().decode()
