"""Pins of the oracle's skip and exponent modes:

- the unit and constant skips of Sec. IV (multiplier a = 1): closed forms
  m_k = m_0 + k b mod n, and the constant-skip symmetry of Eq.
  constantskipsymmetry, (k b)^e = (b^e mod n)(k^e mod n) mod n;
- CRT exponents (the note on large exponents in Sec. V): residue-wise powers,
  m^E mod n for the single exponent E found by a Python CRT when it exists,
  and a permutation of Z_n by brute force on tiny primes.
Expected values come from Python big integers, not from the oracle.
"""
import math
import random

import numpy as np
import pytest

import oracle
import workload

A = 2307085864
Q = (1 << 63) - 25


def _pq(seed):
    p, q, e, ms = oracle.params_from_seed(seed, workload.E_SMALLEST, 3, 3)
    return p, q, e, ms % (p * q)


def messages(p, q, m0, s0, n_out, a=A):
    """m_1..m_N: e = 1 makes the ciphertext the message (Sec. VII's weakened e = 1)."""
    c, _, _, _ = oracle.generate(p, q, 1, m0, s0, n_out, a=a, route=oracle.ROUTE_DIRECT)
    return [int(x) for x in c]


def test_unit_skip_is_counter_mode():
    p, q, e, m0 = _pq(101)
    n = p * q
    N = 3000
    c, r, m1, s1 = oracle.generate(p, q, e, m0, 1, N, a=1)
    for k in range(1, N + 1):
        assert int(c[k - 1]) == pow((m0 + k) % n, e, n)
    assert (m1, s1) == ((m0 + N) % n, 1)
    assert r[0] == oracle.unit(int(c[0]), n)


def test_constant_skip_closed_form_and_symmetry():
    p, q, e, _ = _pq(102)
    n = p * q
    rng = random.Random(5)
    b = rng.randrange(2, Q)
    N = 2000
    c_b, _, _, s_end = oracle.generate(p, q, e, 0, b, N, a=1)
    c_1, _, _, _ = oracle.generate(p, q, e, 0, 1, N, a=1)
    be = pow(b, e, n)
    for k in range(1, N + 1):
        assert int(c_b[k - 1]) == pow(k * b % n, e, n)
        assert int(c_1[k - 1]) == pow(k, e, n)
        assert int(c_b[k - 1]) == be * int(c_1[k - 1]) % n  # Eq. constantskipsymmetry
    assert s_end == b


def python_crt_exponent(p, q, ep, eq):
    a, b = p - 1, q - 1
    g = math.gcd(a, b)
    if (eq - ep) % g:
        return 0
    lcm = a // g * b
    t = ((eq - ep) // g) * pow(a // g, -1, b // g) % (b // g) if b // g > 1 else 0
    E = (ep + a * t) % lcm
    assert E % a == ep % a and E % b == eq % b
    return E


def test_crt_exponent_against_python():
    rng = random.Random(6)
    for seed in range(200, 230):
        p, q, _, _ = _pq(seed)
        for _ in range(20):
            ep = rng.randrange(3, 1 << 16) | 1
            eq = rng.randrange(3, 1 << 16) | 1
            assert oracle.crt_exponent(p, q, ep, eq) == python_crt_exponent(p, q, ep, eq)


def _valid(e, m):
    return math.gcd(e, m) == 1


def test_crt_exponent_stream_equals_large_power():
    rng = random.Random(7)
    found = 0
    for seed in range(300, 400):
        p, q, _, m0 = _pq(seed)
        ep = next(x for x in range(5, 200, 2) if _valid(x, p - 1))
        eq = next(x for x in range(ep + 2, 400, 2) if _valid(x, q - 1))
        E = python_crt_exponent(p, q, ep, eq)
        if E == 0:
            continue
        found += 1
        n = p * q
        N = 500
        c, _, _, _ = oracle.generate(p, q, ep, m0, 1, N, eq=eq)
        for k, mk in enumerate(messages(p, q, m0, 1, N)):
            assert int(c[k]) == pow(mk, E, n)
        if found >= 5:
            break
    assert found >= 3


def test_crt_exponent_stream_without_single_exponent():
    """No E exists: the output is still the Garner combination of the residue powers."""
    for seed in range(400, 500):
        p, q, _, m0 = _pq(seed)
        g = math.gcd(p - 1, q - 1)
        if g < 4:
            continue
        ep = next(x for x in range(3, 200, 2) if _valid(x, p - 1))
        eq = next((x for x in range(3, 400, 2)
                   if _valid(x, q - 1) and (x - ep) % g), None)
        if eq is None:
            continue
        assert python_crt_exponent(p, q, ep, eq) == 0
        N = 400
        c, _, _, _ = oracle.generate(p, q, ep, m0, 1, N, eq=eq)  # checked route
        for k, mk in enumerate(messages(p, q, m0, 1, N)):
            assert int(c[k]) % p == pow(mk % p, ep, p)
            assert int(c[k]) % q == pow(mk % q, eq, q)
        with pytest.raises(RuntimeError):
            oracle.generate(p, q, ep, m0, 1, 4, eq=eq, route=oracle.ROUTE_DIRECT)
        return
    pytest.fail("no prime pair with gcd(p-1, q-1) >= 4 and an inconsistent exponent pair")


def test_crt_exponents_permute_small_rings():
    for p, q in [(11, 23), (7, 13), (5, 17)]:
        n = p * q
        eps = [x for x in range(3, 30, 2) if _valid(x, p - 1)]
        eqs = [x for x in range(3, 30, 2) if _valid(x, q - 1)]
        for ep in eps[:3]:
            for eq in eqs[:3]:
                image = {oracle.crt_encrypt2(m % p, m % q, p, q, ep, eq) for m in range(n)}
                assert image == set(range(n)), (p, q, ep, eq)


def test_equal_exponents_are_the_ordinary_generator():
    p, q, e, m0 = _pq(103)
    c0, r0, m_a, s_a = oracle.generate(p, q, e, m0, 1, 777)
    c1, r1, m_b, s_b = oracle.generate(p, q, e, m0, 1, 777, eq=e)
    np.testing.assert_array_equal(c0, c1)
    assert (m_a, s_a) == (m_b, s_b)


def _exact_want(c, n):
    from fractions import Fraction

    w = float(Fraction(c, n))  # Python rounds a Fraction once, to nearest even
    return 1.0 - 2.0 ** -53 if w >= 1.0 else w


def test_exact_rational_division():
    from fractions import Fraction

    rng = random.Random(8)
    for seed in range(500, 515):
        p, q, _, _ = _pq(seed)
        n = p * q
        cs = [1, 2, 3, n - 1, n - 2, n // 2, n // 3] + [rng.randrange(n) for _ in range(2000)]
        # c/n just below and just above the midpoint of two neighbouring doubles
        for _ in range(300):
            x = rng.random()
            mid = (Fraction(x) + Fraction(math.nextafter(x, 1.0))) / 2
            c = math.floor(mid * n)
            cs += [c, c + 1]
        for c in cs:
            if 0 <= c < n:
                assert oracle.unit_exact(c, n) == _exact_want(c, n), (c, n)


def test_exact_and_paper_readings_differ_often():
    """The two readings of r = c / n disagree in a large share of draws (why the reading
    is pinned)."""
    rng = random.Random(9)
    p, q, _, _ = _pq(600)
    n = p * q
    cs = [rng.randrange(n) for _ in range(20000)]
    diff = sum(oracle.unit(c, n) != oracle.unit_exact(c, n) for c in cs)
    assert diff > 0.1 * len(cs)


def test_vector_call_is_the_interleaved_streams():
    """Eq. vectorize: the Mv-vector update equals the Mv streams interleaved k-major, for
    split substreams (Sec. VI) and for unrelated instances."""
    p, q, e, m0 = _pq(700)
    Mv, N = 8, 501
    s0 = [oracle.split_s0(1, A, Mv, g) for g in range(Mv)]
    pv = np.full(Mv, p, np.uint64)
    qv = np.full(Mv, q, np.uint64)
    ev = np.full(Mv, e, np.uint64)
    av = np.full(Mv, A, np.uint64)
    m = np.full(Mv, m0, np.uint64)
    s = np.array(s0, np.uint64)
    c, r = oracle.generate_vector(pv, qv, ev, av, m, s, N)
    for g in range(Mv):
        cg, rg, mg, sg = oracle.generate(p, q, e, m0, s0[g], N)
        np.testing.assert_array_equal(c[g::Mv], cg)
        np.testing.assert_array_equal(r[g::Mv].view(np.uint64), rg.view(np.uint64))
        assert (int(m[g]), int(s[g])) == (mg, sg)
    # substream 0 continues the parent; substream 1 is the parent shifted by (Q-1)/Mv skips
    assert int(s0[1]) == pow(A, (Q - 1) // Mv, Q)
    # unrelated instances, one with a constant skip
    insts = [_pq(701), _pq(702), _pq(703)]
    pv = np.array([x[0] for x in insts], np.uint64)
    qv = np.array([x[1] for x in insts], np.uint64)
    ev = np.array([x[2] for x in insts], np.uint64)
    av = np.array([A, 1, A], np.uint64)
    m = np.array([x[3] for x in insts], np.uint64)
    s = np.array([1, 99, 1], np.uint64)
    c, _ = oracle.generate_vector(pv, qv, ev, av, m, s, 300)
    for g, (pp, qq, ee, mm) in enumerate(insts):
        cg, _, _, _ = oracle.generate(pp, qq, ee, mm, [1, 99, 1][g], 300, a=int(av[g]))
        np.testing.assert_array_equal(c[g::3], cg)


def test_parallel_seek_equals_serial_seek():
    """The skip sum split over threads (ranges started by jump-ahead) equals the serial walk."""
    for seed, a in ((800, A), (801, 3), (802, 1)):
        p, q, _, m0 = _pq(seed)
        for k in (0, 1, 2, 17, 1000, 123457):
            s0 = 7 if a != 1 else 99
            assert oracle.seek_parallel(p, q, a, m0, s0, k) == oracle.seek(p, q, a, m0, s0, k)
