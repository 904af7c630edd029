"""Pins of the oracle's frequency/serial-test histogram (Sec. VII).

The digit floor(r d) is checked against exact rational arithmetic (Python
Fractions), the tuple counting against a pure-Python rebuild from the
generated sequence, and the power-of-two case against numpy binning (the
scaling by 2^k is exact in binary floating point).
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workload

DS = [2, 10, 16, 100, 1000, 1024, 1 << 20, 10 ** 6, (1 << 31) + 11, (1 << 32) - 1]


def exact_digit(r: float, d: int) -> int:
    return math.floor(Fraction(r) * d)


def test_digit_matches_exact_rational():
    rng = random.Random(7)
    rs = [0.0, 2.0 ** -60, 2.0 ** -1074 * 3, 0.5, 0.1, 0.3, 0.7, 1.0 - 2.0 ** -53]
    rs += [rng.getrandbits(53) / 2.0 ** 53 for _ in range(400)]
    rs += [rng.random() * 2.0 ** -rng.randrange(0, 70) for _ in range(200)]
    for d in DS:
        # values just below and at multiples of 1/d
        for k in range(1, 12):
            x = float(Fraction(k % d, d))
            rs_b = [x, math.nextafter(x, 0.0), math.nextafter(x, 1.0)]
            for r in rs_b:
                if 0.0 <= r < 1.0:
                    assert oracle.digit_of_unit(r, d) == exact_digit(r, d), (r, d)
        for r in rs:
            assert oracle.digit_of_unit(r, d) == exact_digit(r, d), (r, d)


def test_digit_is_the_exact_floor_not_the_rounded_product():
    # 0.3 (as a double) times 10 is 2.99999999999999988898..., which rounds to 3.0.
    assert 0.3 * 10 == 3.0
    assert oracle.digit_of_unit(0.3, 10) == 2
    assert oracle.digit_of_unit(1.0 - 2.0 ** -53, 10) == 9


def _instances(k, seed=11):
    seeds = workload.instance_seeds(seed, k)
    par = [oracle.params_from_seed(int(s), workload.E_UNIFORM, 3, 257) for s in seeds]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    m0 = np.array([int(x[3]) % (int(x[0]) * int(x[1])) for x in par], np.uint64)
    return p, q, e, m0


def python_histogram(c, r, D, d, source):
    """Tuple counting written out in Python from the generated sequence."""
    hist = {}
    ntup = len(c) // D
    for k in range(ntup):
        b = 0
        for i in range(D):
            x = k * D + i
            g = exact_digit(float(r[x]), d) if source == 0 else int(c[x]) % d
            b += g * d ** i
        hist[b] = hist.get(b, 0) + 1
    return hist


@pytest.mark.parametrize("D,d,source", [(1, 1000, 0), (2, 16, 0), (3, 10, 0), (5, 4, 0),
                                        (1, 64, 1), (2, 8, 1), (3, 4, 1)])
def test_histogram_rebuilt_from_sequence(D, d, source):
    p, q, e, m0 = _instances(3)
    a = np.full(3, 2307085864, np.uint64)
    counts = np.array([3001, 1, 4100], np.uint64)
    m = m0.copy()
    s = np.ones(3, np.uint64)
    hist = oracle.histogram_many(p, q, e, a, m, s, counts, D, d, source)
    want = np.zeros(d ** D, np.uint64)
    for i in range(3):
        c, r, _, _ = oracle.generate(int(p[i]), int(q[i]), int(e[i]), int(m0[i]), 1,
                                     int(counts[i]))
        for b, v in python_histogram(c, r, D, d, source).items():
            want[b] += v
    np.testing.assert_array_equal(hist, want)
    assert int(hist.sum()) == sum(int(x) // D for x in counts)
    # the state advanced by the full counts, counted tuples or not
    for i in range(3):
        m1, s1 = oracle.seek(int(p[i]), int(q[i]), 2307085864, int(m0[i]), 1, int(counts[i]))
        assert (int(m[i]), int(s[i])) == (m1, s1)


def test_power_of_two_frequency_matches_numpy_binning():
    p, q, e, m0 = _instances(2, seed=12)
    a = np.full(2, 2307085864, np.uint64)
    counts = np.array([20000, 7777], np.uint64)
    k = 12
    hist = oracle.histogram_many(p, q, e, a, m0.copy(), np.ones(2, np.uint64), counts, 1, 1 << k)
    want = np.zeros(1 << k, np.uint64)
    for i in range(2):
        _, r, _, _ = oracle.generate(int(p[i]), int(q[i]), int(e[i]), int(m0[i]), 1,
                                     int(counts[i]))
        want += np.bincount((r * (1 << k)).astype(np.int64), minlength=1 << k).astype(np.uint64)
    np.testing.assert_array_equal(hist, want)
