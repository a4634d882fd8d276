"""Shared helpers for the GPU parity tests (inputs, transfers, oracle calls)."""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

from paper_2209_01290_gb300 import inputs


def to_dev(x: np.ndarray, device: int = 0):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(f"cuda:{device}")


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def operands(seed: int, qs, npoly: int, n: int):
    return inputs.operand_pair(seed, qs, npoly, n)


def oracle_polymul_batch(oracle, a: np.ndarray, b: np.ndarray, qs, psis, threads: int = 0):
    """Oracle product of every unit of [P][L][N] operands (scalar NTT; the
    schoolbook for N <= 1024)."""
    P, L, N = a.shape
    a2, b2 = a.reshape(P * L, N), b.reshape(P * L, N)
    threads = threads or min(16, os.cpu_count() or 1)

    def one(u):
        l = u % L
        return oracle.polymul(a2[u], b2[u], int(qs[l]), int(psis[l]))

    with cf.ThreadPoolExecutor(threads) as ex:
        out = list(ex.map(one, range(P * L)))
    return np.stack(out).reshape(P, L, N)


def schoolbook_coeff(a: np.ndarray, b: np.ndarray, q: int, k: int) -> int:
    """c_k of the negacyclic product by its definition, in Python integers."""
    n = a.size
    ai = np.array([int(x) for x in a], dtype=object)
    bi = np.array([int(x) for x in b], dtype=object)
    pos = int(np.dot(ai[: k + 1], bi[k::-1])) if k >= 0 else 0
    neg = int(np.dot(ai[k + 1:], bi[n - 1:k:-1])) if k + 1 < n else 0
    return (pos - neg) % q
