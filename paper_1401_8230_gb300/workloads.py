"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

These generate the request sets of the batched and serving benchmarks from numpy's PCG64
generator with fixed seeds. Tests feed the same parameters to the CUDA library and to the
CPU oracle, so both sides see identical inputs.
"""
from __future__ import annotations

import numpy as np


def log_uniform_lengths(rng: np.random.Generator, n: int, lo: int, hi: int) -> np.ndarray:
    """n integer lengths, log-uniform on [lo, hi]."""
    x = rng.uniform(np.log(lo), np.log(hi), size=n)
    return np.clip(np.round(np.exp(x)).astype(np.int64), lo, hi)


def batched_requests(n: int = 4096, lo: int = 2**8, hi: int = 2**26, seed: int = 1, chunk: int = 1024):
    """The batched workload: n requests with log-uniform lengths in [lo, hi], each with its own
    uniform 64-bit seed and a stream offset (cumulative stream count, so streams never repeat
    within a seed family). Returns a list of dicts (length, seed, first_stream, chunk)."""
    rng = np.random.default_rng(seed)
    lengths = log_uniform_lengths(rng, n, lo, hi)
    seeds = rng.integers(0, 2**63, size=n, dtype=np.uint64) * 2 + rng.integers(0, 2, size=n, dtype=np.uint64)
    out, first = [], 0
    for L, s in zip(lengths, seeds):
        out.append({"length": int(L), "seed": int(s), "first_stream": first, "chunk": chunk})
        first += (int(L) + chunk - 1) // chunk
    return out


def serving_arrivals(duration_s: float, rate_hz: float = 20000.0, lo: int = 2**10, hi: int = 2**28,
                     n_clients: int = 2**16, seed: int = 1):
    """Poisson arrivals at rate_hz over duration_s: (arrival time, client, length, form) with
    log-uniform lengths in [lo, hi] and the form drawn uniformly from {A, B, C}."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate_hz * duration_s))
    times = np.sort(rng.uniform(0.0, duration_s, size=n))
    clients = rng.integers(0, n_clients, size=n)
    lengths = log_uniform_lengths(rng, n, lo, hi)
    forms = rng.integers(0, 3, size=n)
    return [{"t": float(t), "client": int(c), "length": int(L), "form": int(f)}
            for t, c, L, f in zip(times, clients, lengths, forms)]
