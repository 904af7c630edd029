"""Hard inputs for the output step r = RN(RN(c) / RN(n)) (Sec. V, Eq. CodeFloatingPointStep).

A division route can only go wrong where the quotient of the two converted
operands lies very close to a midpoint between neighbouring doubles: there a
quotient approximation with a tiny error rounds the other way. Random
ciphertexts almost never land there (the quotient's distance to a midpoint is
then about 2^-53 relative), so these inputs are built to land there on
purpose.

Construction. Write RN(n) = b 2^eN and RN(c) = a 2^eC with integer
significands a, b in [2^52, 2^53). A midpoint between doubles of the binade
of a/b has an odd 54-bit significand m': a/b = m' 2^-53 + t 2^-53 / b when
a >= b, a/b = m' 2^-54 + t 2^-54 / b when a < b, for an integer t. For a
chosen small t the equation a 2^K - m' b = t (K = 53 or 54) fixes m' modulo
2^(K - j) (b = 2^j b_odd, t a multiple of 2^j with an odd cofactor, which
makes m' odd), and then a = (m' b + t) / 2^K. So a / b lies |t| / (b 2^K)
from the midpoint m' 2^-K: for |t| = 1 that is within 2^-106 relative, the
closest a quotient of two doubles can come to a midpoint. Each such a is
used at every exponent eC with RN(c) = a 2^eC <= RN(n), and for eC > 0 with
several integers c that round to that double (the centre, its neighbours,
the interval's ends and ties, and random interior points), so that the
conversion of c (exact below 2^53, rounded above) is exercised as well.

This module only builds inputs; the expected outputs come from the oracle
(and, in the CPU pins, from Python's correctly rounded integer division).
"""
from __future__ import annotations

import math

import numpy as np

# Test moduli n = p q (primes in [2^31, 2^32)) at the edges of the modulus range,
# chosen so that the odd-significand construction gives the closest cases:
# (p, q, what the modulus exercises)
EDGE_MODULI = [
    (2147483659, 2147483713, "n just above 2^62, RN(n) with an odd significand"),
    (3037000453, 3037000537, "n just below 2^63 (near Q), significand of RN(n) near 2"),
    (3037001507, 3036999499, "n just above 2^63 (near Q), significand of RN(n) near 1"),
    (4294967279, 4294967231, "n just below 2^64, odd significand near 2"),
    (4294967291, 4294967279, "the largest n, RN(n) significand divisible by 2^22"),
]


def split_double(x: float) -> tuple[int, int]:
    """(significand, exponent) with x = significand * 2^exponent, significand in [2^52, 2^53)."""
    m, e = math.frexp(x)
    return int(m * (1 << 53)), e - 53


def _near_midpoint_significands(b: int, t_max: int, rng: np.random.Generator,
                                per_t: int = 2) -> list[int]:
    """Significands a in [2^52, 2^53) with a / b within (t_max 2^j) / (b 2^53) of a midpoint."""
    j = (b & -b).bit_length() - 1
    bo = b >> j
    out = []
    for K in (53, 54):
        mod = 1 << (K - j)
        inv = pow(bo, -1, mod)
        for to in range(-t_max, t_max + 1, 2):  # odd cofactors
            r = (-to * inv) % mod
            # candidates m' = r + i mod in (2^53, 2^54); sample a few when there are many
            lo = max(0, -((r - (1 << 53)) // mod))
            hi = ((1 << 54) - 1 - r) // mod
            if hi < lo:
                continue
            cnt = hi - lo + 1
            picks = range(lo, hi + 1) if cnt <= per_t else \
                sorted(set(int(x) for x in rng.integers(lo, hi + 1, per_t)))
            for i in picks:
                mp = r + i * mod
                num = mp * b + (to << j)
                assert num % (1 << K) == 0 and mp & 1
                a = num >> K
                if not (1 << 52) <= a < (1 << 53):
                    continue
                if (K == 53) != (a >= b):  # the binade the midpoint was taken in
                    continue
                out.append(a)
    return out


def near_midpoint_ciphertexts(n: int, t_max: int = 3071, seed: int = 0,
                              interior: int = 2) -> np.ndarray:
    """Ciphertexts c < n whose RN(c)/RN(n) lies next to a midpoint between doubles."""
    rng = np.random.default_rng(seed)
    b, eN = split_double(float(n))
    out = set()
    for a in _near_midpoint_significands(b, t_max, rng):
        for eC in range(0, eN + 2):
            C = a << eC
            if C > n + (1 << eN):
                break
            if eC == 0:
                cands = [C]
            else:
                h = 1 << (eC - 1)
                cands = [C, C - 1, C + 1, C - h + 1, C + h - 1, C - h, C + h]
                if h > 2:
                    cands += [C - h + 1 + int(x) for x in rng.integers(0, 2 * h - 1, interior,
                                                                        dtype=np.uint64)]
            out.update(c for c in cands if 0 <= c < n)
    return np.array(sorted(out), dtype=np.uint64)


def reference_unit(c: int, n: int) -> float:
    """RN(RN(c)/RN(n)) with the 1.0 guard, from Python's correctly rounded int division.

    float(int) rounds to nearest even and int / int is correctly rounded, so
    this does not use the hardware's double division.
    """
    r = int(float(c)) / int(float(n))
    return 1.0 - 2.0 ** -53 if r >= 1.0 else r


def midpoint_distance_ulps(c: int, n: int) -> float:
    """|RN(c)/RN(n) - nearest midpoint| in units of the quotient's ulp (exact rational)."""
    from fractions import Fraction

    x = Fraction(int(float(c)), int(float(n)))
    if x == 0:
        return 0.5
    e = math.floor(math.log2(x))
    if Fraction(2) ** e > x:
        e -= 1
    elif Fraction(2) ** (e + 1) <= x:
        e += 1
    ulp = Fraction(2) ** (e - 52)
    k = math.floor(x / ulp)
    mid = (k + Fraction(1, 2)) * ulp
    return float(abs(x - mid) / ulp)
