"""Exact negacyclic polynomial multiplication on GB300 (sm_103a).

c = a * b in Z_q[X]/(X^N + 1) computed as in arxiv 2209.01290, Eq. 2: merged
Cooley-Tukey forward NTT (Algorithm 6), pointwise product with the Barrett
variant of Algorithm 4, merged Gentleman-Sande inverse NTT (Algorithm 7) with
the 1/N scaling folded in (into the last inverse stage by default, or as a 1/2
at every inverse butterfly with ``halving=True``).  All arithmetic runs in the CUDA
library built from ``csrc/`` (C ABI in ``include/pm.h``); this package only
marshals torch tensors (device memory, streams) into that ABI.

Tensors are int64 (or uint64) with values in [0, q_l), shaped
[npoly, nlimbs, N] (or anything with that many contiguous elements).
"""
from __future__ import annotations

from . import capi
from .capi import PMError, pm_find_params  # noqa: F401

__all__ = ["Plan", "Queue", "find_params", "PMError", "capi"]


def find_params(n: int, nlimbs: int = 1, qbits: int = 60):
    """(q list, psi list): the nlimbs largest primes q < 2^qbits, q = 1 mod 2N."""
    return pm_find_params(_log2(n), nlimbs, qbits)


def _log2(n: int) -> int:
    if n < 2 or n & (n - 1):
        raise ValueError(f"N={n} must be a power of two >= 2")
    return n.bit_length() - 1


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A device-resident plan for one (N, {q_l}, {psi_l})."""

    def __init__(self, n: int, qs, psis=None, device: int = 0, halving: bool = False,
                 fused: bool = False, word32: bool = False):
        """halving=True scales by 1/2 at every inverse butterfly (the paper's
        Eq. 2 form); the default folds 1/N into the last inverse stage.
        fused=True computes products by Algorithm 8 (N >= 4).
        word32=True: 32-bit words (every q < 2^30); the tensors are int32
        (bit patterns of uint32) instead of int64."""
        self.n = n
        self.log2n = _log2(n)
        self.device = device
        self.word32 = word32
        flags = ((capi.PM_PLAN_HALVING if halving else 0) | (capi.PM_PLAN_FUSED if fused else 0)
                 | (capi.PM_PLAN_WORD32 if word32 else 0))
        self._h = capi.pm_plan_create_ex(self.log2n, list(qs), psis, device, flags)
        _, self.nlimbs, self.qs, self.psis = capi.pm_plan_info(self._h)

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            capi.pm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    # -- argument checks (the C side re-checks pointers and sizes)
    def _npoly(self, t) -> int:
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected a CUDA tensor")
        want = (torch.int32,) if self.word32 else (torch.int64, torch.uint64)
        if t.dtype not in want:
            raise TypeError(f"expected {'int32' if self.word32 else 'int64/uint64'}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if t.device.index != self.device:
            raise ValueError(f"tensor on cuda:{t.device.index}, plan on cuda:{self.device}")
        per = self.nlimbs * self.n
        if t.numel() == 0 or t.numel() % per:
            raise ValueError(f"numel {t.numel()} is not a positive multiple of nlimbs*N = {per}")
        return t.numel() // per

    # -- hot path
    def ntt_fwd_(self, x, stream=None):
        npoly = self._npoly(x)
        fn = capi.pm_ntt_fwd32 if self.word32 else capi.pm_ntt_fwd
        fn(self.handle, x.data_ptr(), npoly, _stream_handle(stream))
        return x

    def ntt_inv_(self, x, stream=None):
        npoly = self._npoly(x)
        fn = capi.pm_ntt_inv32 if self.word32 else capi.pm_ntt_inv
        fn(self.handle, x.data_ptr(), npoly, _stream_handle(stream))
        return x

    def pointwise(self, a, b, out=None, stream=None):
        import torch
        npoly = self._npoly(a)
        if self._npoly(b) != npoly:
            raise ValueError("a and b differ in size")
        out = torch.empty_like(a) if out is None else out
        if self._npoly(out) != npoly:
            raise ValueError("out has the wrong size")
        fn = capi.pm_pointwise32 if self.word32 else capi.pm_pointwise
        fn(self.handle, a.data_ptr(), b.data_ptr(), out.data_ptr(), npoly, _stream_handle(stream))
        return out

    def polymul(self, a, b, out=None, stream=None):
        import torch
        npoly = self._npoly(a)
        if self._npoly(b) != npoly:
            raise ValueError("a and b differ in size")
        out = torch.empty_like(a) if out is None else out
        if self._npoly(out) != npoly:
            raise ValueError("out has the wrong size")
        fn = capi.pm_polymul32 if self.word32 else capi.pm_polymul
        fn(self.handle, a.data_ptr(), b.data_ptr(), out.data_ptr(), npoly, _stream_handle(stream))
        return out

    def polymul_host(self, h_a, h_b, h_c, d_a, d_b, d_c, stream=None):
        """Host-to-host product through device buffers (copies pipelined)."""
        npoly = self._npoly(d_a)
        for h in (h_a, h_b, h_c):
            if h.is_cuda or not h.is_contiguous() or h.numel() != d_a.numel():
                raise ValueError("host tensors must be contiguous CPU tensors of the same size")
        capi.pm_polymul_host(self.handle, h_a.data_ptr(), h_b.data_ptr(), h_c.data_ptr(),
                             d_a.data_ptr(), d_b.data_ptr(), d_c.data_ptr(), npoly,
                             _stream_handle(stream))
        return h_c

    def reserve(self, npoly: int, stream=None) -> None:
        capi.pm_plan_reserve(self.handle, npoly, _stream_handle(stream))

    def graph_polymul(self, a, b, c) -> "Graph":
        """Capture c = a * b into a CUDA graph (replay with Graph.launch)."""
        npoly = self._npoly(a)
        if self._npoly(b) != npoly or self._npoly(c) != npoly:
            raise ValueError("a, b, c differ in size")
        return Graph(capi.pm_graph_create_polymul(self.handle, a.data_ptr(), b.data_ptr(),
                                                  c.data_ptr(), npoly), self.device)

    def check_reduced(self, x, stream=None) -> bool:
        npoly = self._npoly(x)
        fn = capi.pm_check_reduced32 if self.word32 else capi.pm_check_reduced
        return fn(self.handle, x.data_ptr(), npoly, _stream_handle(stream))

    def sync(self, stream=None) -> None:
        capi.pm_plan_sync(self.handle, _stream_handle(stream))


class Graph:
    """A captured polymul (pm_graph_create_polymul)."""

    def __init__(self, handle: int, device: int):
        self._h = handle
        self.device = device

    def launch(self, stream=None) -> None:
        capi.pm_graph_launch(self._h, _stream_handle(stream))

    def close(self) -> None:
        if getattr(self, "_h", None):
            capi.pm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Queue:
    """Reusable context for uneven batches (pm_polymul_uneven)."""

    def __init__(self, device: int = 0, mode: int = 0):
        """mode: capi.PM_UNEVEN_AUTO (0), _PERSISTENT (1) or _GROUPED (2)."""
        self.device = device
        self._h = capi.pm_queue_create(device)
        if mode:
            capi.pm_queue_set_mode(self._h, mode)

    def close(self) -> None:
        if getattr(self, "_h", None):
            capi.pm_queue_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, units: int, scratch_words: int) -> None:
        capi.pm_queue_reserve(self._h, units, scratch_words)

    def polymul_uneven(self, jobs, stream=None) -> None:
        """jobs: list of (Plan, a, b, c) with CUDA tensors shaped for the plan."""
        raw = []
        for plan, a, b, c in jobs:
            npoly = plan._npoly(a)
            if plan._npoly(b) != npoly or plan._npoly(c) != npoly:
                raise ValueError("a, b, c differ in size")
            raw.append((plan.handle, a.data_ptr(), b.data_ptr(), c.data_ptr(), npoly))
        capi.pm_polymul_uneven(self._h, raw, _stream_handle(stream))

    def sync(self, stream=None) -> None:
        capi.pm_queue_sync(self._h, _stream_handle(stream))
