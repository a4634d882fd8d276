"""Seeded synthetic inputs for negacyclic polynomial multiplication.

This module holds no arithmetic of the method: it only draws coefficients
uniformly from [0, q) (Sec. II-B: operands and moduli "randomly sampled from a
uniform distribution") and describes workload shapes.  It is the one piece
shared by the GPU path's tests/bench and the CPU oracle; moduli are passed in
by the caller.

Generator: numpy's PCG64 bit generator seeded with ``seed``; coefficients of
limb l are ``Generator.integers(0, q_l, dtype=uint64)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 0x220901290


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_mod(g: np.random.Generator, q: int, shape) -> np.ndarray:
    """i.i.d. uniform integers in [0, q) as uint64."""
    return g.integers(0, q, size=shape, dtype=np.uint64)


def uniform_limbs(seed: int, qs, npoly: int, n: int) -> np.ndarray:
    """Array [npoly][L][n] with limb l uniform in [0, qs[l])."""
    g = rng(seed)
    L = len(qs)
    out = np.empty((npoly, L, n), dtype=np.uint64)
    for p in range(npoly):
        for l, q in enumerate(qs):
            out[p, l] = uniform_mod(g, int(q), n)
    return out


def uniform_limbs_torch(seed: int, qs, npoly: int, n: int, device="cuda"):
    """Device-side version of uniform_limbs for large batches: int64 tensor
    [npoly][L][n], limb l uniform in [0, qs[l]) (torch's seeded generator;
    a different stream of numbers than the numpy generator)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((npoly, len(qs), n), dtype=torch.int64, device=device)
    for l, q in enumerate(qs):
        out[:, l, :] = torch.randint(0, int(q), (npoly, n), generator=g, device=device,
                                     dtype=torch.int64)
    return out


def operand_pair(seed: int, qs, npoly: int, n: int):
    """(a, b), each [npoly][L][n], independent uniform draws."""
    a = uniform_limbs(seed, qs, npoly, n)
    b = uniform_limbs(seed ^ 0x5A5A5A5A, qs, npoly, n)
    return a, b


@dataclass(frozen=True)
class UnevenJobShape:
    log2n: int
    nlimbs: int


def uneven_shapes(seed: int, njobs: int = 512, log2n_range=(12, 17),
                  max_limbs: int = 48) -> list[UnevenJobShape]:
    """Uneven batch: N uniform over {2^lo..2^hi}, limb count uniform in 1..max_limbs."""
    g = rng(seed)
    lo, hi = log2n_range
    ln = g.integers(lo, hi + 1, size=njobs)
    ll = g.integers(1, max_limbs + 1, size=njobs)
    return [UnevenJobShape(int(a), int(b)) for a, b in zip(ln, ll)]


@dataclass(frozen=True)
class Request:
    arrival_s: float
    log2n: int
    nlimbs: int


def poisson_requests(seed: int, rate_hz: float, duration_s: float,
                     log2n_choices=(13, 15, 16), weights=(0.3, 0.4, 0.3),
                     max_limbs: int = 32, limit: int | None = None) -> list[Request]:
    """Poisson arrivals (exponential gaps) with N drawn from `log2n_choices`
    by `weights` and limb count uniform in 1..max_limbs."""
    g = rng(seed)
    reqs: list[Request] = []
    t = 0.0
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    while True:
        t += float(g.exponential(1.0 / rate_hz))
        if t >= duration_s or (limit is not None and len(reqs) >= limit):
            break
        ln = int(g.choice(np.asarray(log2n_choices), p=w))
        reqs.append(Request(t, ln, int(g.integers(1, max_limbs + 1))))
    return reqs


def expected_request_bytes(log2n_choices=(13, 15, 16), weights=(0.3, 0.4, 0.3),
                           max_limbs: int = 32) -> float:
    """Mean operand+result bytes of one request (a, b, c of uint64)."""
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    mean_n = float(sum(wi * (1 << ln) for wi, ln in zip(w, log2n_choices)))
    return 24.0 * mean_n * (1 + max_limbs) / 2.0


def seed_for(config_index: int) -> int:
    return SEED_BASE + config_index


def log2(n: int) -> int:
    if n < 1 or n & (n - 1):
        raise ValueError(f"{n} is not a power of two")
    return int(math.log2(n))
