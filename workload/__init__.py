"""Seeded synthetic inputs shared by the GPU library's tests/bench and the oracle.

This module holds none of the generator's arithmetic: it only draws seeds,
stream lengths and request traces. Everything is a pure function of a master
seed, so both sides of a parity test see the same inputs.

Per-instance seeds are SplitMix64 outputs (Steele, Lea & Flood 2014) of the
master stream: seed_i = mix(master + (i + 1) * 0x9E3779B97F4A7C15). Each side
turns a seed into (p, q, e, message seed) with its own SplitMix64 and
primality test, following the rule documented at the library's
``rsaprng_params_from_seed`` and the oracle's ``or_params_from_seed``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Exponent rules (same numbering on both sides).
E_SMALLEST, E_UNIFORM, E_AT_LEAST = 0, 1, 2


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(master: int, count: int, first: int = 0) -> np.ndarray:
    """Outputs first..first+count-1 of SplitMix64 started at `master`."""
    with np.errstate(over="ignore"):
        k = np.arange(first + 1, first + count + 1, dtype=np.uint64)
        return _mix(np.uint64(master) + k * GAMMA)


def instance_seeds(master: int, count: int, first: int = 0) -> np.ndarray:
    """Per-instance 64-bit seeds for instances first..first+count-1."""
    return splitmix64(master, count, first)


def uniform01(master: int, count: int, first: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64 draws."""
    return (splitmix64(master, count, first) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def lognormal_lengths(master: int, count: int, median: float = 2.0**14, sigma: float = 1.388,
                      lo: int = 100, hi: int = 10_000_000) -> np.ndarray:
    """Stream lengths ~ lognormal(ln median, sigma), rounded and clipped to [lo, hi].

    Normals come from a Box-Muller transform of SplitMix64 uniforms, so the
    lengths depend only on the master seed.
    """
    u1 = uniform01(master, count, 0)
    u2 = uniform01(master ^ 0x5DEECE66D, count, 0)
    u1 = np.maximum(u1, 2.0**-53)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    x = np.exp(np.log(median) + sigma * z)
    return np.clip(np.rint(x), lo, hi).astype(np.uint64)


def poisson_arrivals(master: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    u = np.maximum(uniform01(master, count, 0), 2.0**-53)
    return np.cumsum(-np.log(u) / rate_per_s)


def loguniform_counts(master: int, count: int, lo: int = 2**4, hi: int = 2**24) -> np.ndarray:
    """Request sizes log-uniform on [lo, hi] (integers)."""
    u = uniform01(master, count, 0)
    x = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.floor(x), lo, hi).astype(np.uint64)


def uniform_indices(master: int, count: int, n: int) -> np.ndarray:
    """Uniform instance indices in [0, n) (multiply-shift of the top 32 bits)."""
    hi32 = splitmix64(master, count, 0) >> np.uint64(32)
    return ((hi32 * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


# Named workloads. Each maps to the sizes the paper's method is exercised at.
CONFIGS = {
    "plain_1x1e6": dict(master=1, instances=1, count=1_000_000, e_rule=E_SMALLEST,
                        e_lo=3, e_hi=3, outputs="u64+f64"),
    "bulk_1024x2^20": dict(master=2, instances=1024, count=1 << 20, e_rule=E_UNIFORM,
                           e_lo=3, e_hi=65537, outputs="f64"),
    "split_65536x32x2^16": dict(master=3, instances=65536, substreams=32, count=1 << 16,
                                e_rule=E_AT_LEAST, e_lo=3, e_hi=3, outputs="u64+f64"),
    "batched_1e5_lognormal": dict(master=4, instances=100_000, e_rule=E_UNIFORM, e_lo=3,
                                  e_hi=257, outputs="f64"),
    "serving_1e6": dict(master=5, instances=1_000_000, e_rule=E_SMALLEST, e_lo=3, e_hi=3,
                        outputs="f64"),
}
