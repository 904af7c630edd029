"""The reciprocal division route of the output step, checked exhaustively at small precision.

Sec. V, Eq. CodeFloatingPointStep: r = RN(C / N) with C = RN(c), N = RN(n).
The library's default route computes it without a division: y = RN(1/N)
(once per instance, on the host), q0 = RN(C y), r = RN(C - q0 N) (one fused
multiply-add) and the result RN(q0 + r y) (a second one). The argument that
this always equals RN(C / N) does not depend on the precision p of the
binary format (only on u = 2^-p and on the significands lying in [1, 2)),
so it can be checked over every pair of significands at small p, with exact
integer arithmetic standing in for each rounded operation. Exponents only
scale every step by the same power of two (no underflow or overflow occurs
for c < n < 2^64), so significand pairs are the whole input space.

The check also counts the pairs whose first quotient q0 is not a faithful
rounding of C / N (it can be 1.5 units off when C's significand is below
N's), so that the test exercises the case in which the classical form of
Markstein's theorem does not apply directly.
"""
import pytest


def _round(m, e, p, sticky=False):
    """RN of (m + s) 2^e to p bits, ties to even; m >= 0 integer, s in (0, 1) iff sticky.

    Returns (significand, exponent) with the significand in [2^(p-1), 2^p), or (0, 0).
    """
    if m == 0:
        return (0, 0)
    shift = m.bit_length() - p
    if shift <= 0:
        assert not sticky
        return (m << -shift, e + shift)
    q = m >> shift
    rem = m & ((1 << shift) - 1)
    half = 1 << (shift - 1)
    if rem > half or (rem == half and (sticky or q & 1)):
        q += 1
    elif rem == half and not sticky and not q & 1:
        pass
    if q >> p:
        q >>= 1
        shift += 1
    return (q, e + shift)


def _round_ratio(num, den, p):
    """RN(num / den) to p bits for positive integers."""
    shift = p + 2 - (num.bit_length() - den.bit_length())
    q, r = divmod(num << shift, den)
    return _round(q, -shift, p, r != 0)


def _round_signed(m, e, p):
    s, (q, ee) = (-1 if m < 0 else 1), _round(abs(m), e, p)
    return s * q, ee


def _add(m1, e1, m2, e2):
    """Exact sum of m1 2^e1 and m2 2^e2 as (m, e)."""
    e = min(e1, e2)
    return (m1 << (e1 - e)) + (m2 << (e2 - e)), e


def _reciprocal_route(a, b, p):
    """RN(q0 + RN(A - B q0) y) for A = a 2^(1-p), B = b 2^(1-p); returns (result, q0 faithful)."""
    Y, ey = _round_ratio(1 << (p - 1), b, p)              # y = RN(1/B)
    Q0, eq = _round(a * Y, ey - (p - 1), p)                 # q0 = RN(A y)
    m, e = _add(a, 1 - p, -(b * Q0), eq + 1 - p)            # A - B q0, exact
    R, er = _round_signed(m, e, p)                          # one FMA
    v, ev = _add(Q0, eq, R * Y, er + ey)                    # q0 + r y, exact
    assert v > 0
    res = _round(v, ev, p)                                  # the second FMA
    # faithful: |q0 - a/b| < ulp(a/b), i.e. |Q0 2^eq b - a 2^0| < 2^(ex + 1 - p) b
    ex = 0 if a >= b else -1
    lhs, el = _add(b * Q0, eq, -a, 0)
    faithful = abs(lhs) * 2 ** (el - (ex + 1 - p)) < b
    return res, faithful


@pytest.mark.parametrize("p", [6, 7, 8, 9, 10, 11])
def test_reciprocal_route_is_correctly_rounded_for_every_significand_pair(p):
    lo, hi = 1 << (p - 1), 1 << p
    unfaithful = 0
    for a in range(lo, hi):
        for b in range(lo, hi):
            got, faithful = _reciprocal_route(a, b, p)
            assert got == _round_ratio(a, b, p), (p, a, b)
            unfaithful += not faithful
            if not faithful:
                assert a < b  # only below 1, as the error bound says
    assert unfaithful > 0  # the 1.5-unit case occurs and is still rounded correctly


def test_rounding_helper_against_python_floats():
    """At p = 53 the helper is IEEE double rounding: compare with Python's int / int."""
    import random

    rng = random.Random(5)
    for _ in range(20000):
        a = rng.randrange(1, 1 << 64)
        b = rng.randrange(1, 1 << 64)
        q, e = _round_ratio(a, b, 53)
        assert q * 2.0**e == a / b
