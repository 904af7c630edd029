"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU),
builds it, and runs the pin checks against that copy: at least one check
must fail. The checks restate the pins of test_oracle_pins.py against raw C
entry points so they can run on any build of the oracle.
"""
import ctypes
import math
import os
import random
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "rsaprng_oracle.c")
Q = (1 << 63) - 25
A = 2307085864


class P(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint64), ("q", ctypes.c_uint64), ("e", ctypes.c_uint64),
                ("a", ctypes.c_uint64), ("Q", ctypes.c_uint64), ("eq", ctypes.c_uint64)]


def _gen(L, p, q, e, m0, s0, n, a=A, qm=Q, route=0):
    prm = P(p, q, e, a, qm)
    m, s = ctypes.c_uint64(m0), ctypes.c_uint64(s0)
    c = np.empty(n, np.uint64)
    r = np.empty(n, np.float64)
    rc = L.or_generate(ctypes.byref(prm), ctypes.byref(m), ctypes.byref(s), n,
                       c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                       r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), route)
    return rc, c, r, m.value, s.value


def _sieve(lo, hi):
    seg = np.ones(hi - lo, bool)
    for d in range(2, int(math.isqrt(hi)) + 1):
        start = max(d * d, (lo + d - 1) // d * d)
        seg[start - lo::d] = False
    return set((lo + np.nonzero(seg)[0]).tolist())


PRIMES_WIN = None


def check_primality(L):
    global PRIMES_WIN
    lo = 1 << 31
    if PRIMES_WIN is None:
        PRIMES_WIN = _sieve(lo, lo + (1 << 14))
    if any(L.or_is_prime(x) for x in (2047, 1373653, 25326001, 3215031751, 2152302898747,
                                       3474749660383, 341550071728321, 3825123056546413051)):
        return False
    if not L.or_is_prime(Q):
        return False
    return all(bool(L.or_is_prime(x)) == (x in PRIMES_WIN) for x in range(lo + 1, lo + (1 << 14), 2))


def check_roots(L):
    fs = [2, 3, 17, 23, 319279, 456065899]
    prim = [g for g in range(2, 12)
            if L.or_powmod(g, Q - 1, Q) == 1 and all(L.or_powmod(g, (Q - 1) // f, Q) != 1 for f in fs)]
    return prim == [3, 6, 7, 10, 11]


def check_skips(L):
    rng = random.Random(1)
    for a in (A, 3157107955, 3, 11):
        for _ in range(300):
            s = rng.randrange(1, Q)
            if L.or_skip_next_schrage(s, a, Q) != a * s % Q or L.or_skip_next_direct(s, a, Q) != a * s % Q:
                return False
    return True


def check_period_tiny_q(L):
    qp, a, p, q = 47, 5, 5, 11
    n, per = p * q, 46 * 55
    rc, c, _, _, _ = _gen(L, p, q, 1, 7, 1, 2 * per, a=a, qm=qp)
    if rc != 0:
        return False
    msgs = [int(x) for x in c]
    b = qp * (qp - 1) // 2
    counts = np.bincount(np.array(msgs[:per]), minlength=n)
    return (counts == qp - 1).all() and all(msgs[k + qp - 1] == (msgs[k] + b) % n for k in range(per))


def check_closed_form(L):
    p, q, e = 2147483659, 2147483693, 5
    n = p * q
    rc, c, r, m_end, s_end = _gen(L, p, q, e, 12345, 1, 200)
    if rc != 0:
        return False
    acc = 12345
    for k in range(1, 201):
        acc = (acc + pow(A, k, Q)) % n
        if int(c[k - 1]) != pow(acc, e, n):
            return False
    return m_end == acc and s_end == pow(A, 200, Q)


def check_rsa(L):
    rng = random.Random(2)
    p, q = 4294967291, 4294967279
    n = p * q
    qinv = pow(q, -1, p)
    for e in (5, 7, 65537):
        if math.gcd(e, (p - 1) * (q - 1)) != 1:
            continue
        d = pow(e, -1, (p - 1) * (q - 1))
        for m in [0, 1, n - 1] + [rng.randrange(n) for _ in range(100)]:
            c = L.or_encrypt_direct(m, e, n)
            if c != pow(m, e, n) or pow(c, d, n) != m:
                return False
            if L.or_crt_encrypt(m % p, m % q, p, q, e, qinv) != c:
                return False
            if L.or_crt_encrypt(m % q, m % p, q, p, e, pow(p, -1, q)) != c:
                return False
    return True


def check_unit(L):
    rng = random.Random(3)
    for n in (4294967291 * 4294967279, 2147483659 * 2147483693):
        for c in [0, 1, n - 1, n - 2] + [rng.randrange(n) for _ in range(2000)]:
            want = float(Fraction(float(c)) / Fraction(float(n)))
            want = 0.9999999999999999 if want >= 1.0 else want
            if L.or_unit(c, n) != want:
                return False
    return True


def check_split(L):
    return all(L.or_split_s0(1, A, Q, mv, g) == pow(A, g * ((Q - 1) // mv), Q)
               for mv in (2, 32, 1000) for g in (0, 1, mv - 1))


def check_histogram(L):
    # digits: exact floor(r d), e.g. 0.3 * 10 rounds to 3.0 but its floor is 2
    for r, d in [(0.3, 10), (0.1, 10), (1 - 2.0 ** -53, 10), (0.7, 1000), (0.5, 1 << 20)]:
        if L.or_digit_of_unit(r, d) != math.floor(Fraction(r) * d):
            return False
    # D = 2 tuples of a short sequence, rebuilt in Python
    p, q, e, N, D, d = 2147483659, 2147483693, 5, 101, 2, 8
    rc, c, r, _, _ = _gen(L, p, q, e, 777, 1, N)
    if rc != 0:
        return False
    want = np.zeros(d ** D, np.uint64)
    for k in range(N // D):
        want[sum(math.floor(Fraction(float(r[k * D + i])) * d) * d ** i for i in range(D))] += 1
    prm = P(p, q, e, A, Q)
    m, s = ctypes.c_uint64(777), ctypes.c_uint64(1)
    hist = np.zeros(d ** D, np.uint64)
    if L.or_histogram(ctypes.byref(prm), ctypes.byref(m), ctypes.byref(s), N, D, d, 0, 0,
                      hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))) != 0:
        return False
    return bool((hist == want).all())


def _crt_e(p, q, ep, eq):
    a, b = p - 1, q - 1
    g = math.gcd(a, b)
    if (eq - ep) % g:
        return 0
    t = ((eq - ep) // g) * pow(a // g, -1, b // g) % (b // g) if b // g > 1 else 0
    return (ep + a * t) % (a // g * b)


def check_modes(L):
    p, q, e = 2147483659, 2147483693, 5
    n = p * q
    # unit skip (a = 1): counter mode m_k = m_0 + k
    rc, c, _, _, _ = _gen(L, p, q, e, 123, 1, 50, a=1)
    if rc != 0 or any(int(c[k - 1]) != pow((123 + k) % n, e, n) for k in range(1, 51)):
        return False
    # CRT exponents: residue-wise powers and the single exponent
    ep = next(x for x in range(3, 99, 2) if math.gcd(x, p - 1) == 1)
    eq = next(x for x in range(ep + 2, 199, 2) if math.gcd(x, q - 1) == 1)
    if L.or_crt_exponent(p, q, ep, eq) != _crt_e(p, q, ep, eq):
        return False
    inv = pow(q, -1, p)
    rng = random.Random(9)
    for m in [0, 1, n - 1] + [rng.randrange(n) for _ in range(50)]:
        c = L.or_crt_encrypt2(m % p, m % q, p, q, ep, eq, inv)
        if c % p != pow(m % p, ep, p) or c % q != pow(m % q, eq, q) or c >= n:
            return False
    return True


def check_unit_exact(L):
    rng = random.Random(10)
    for n in (4294967291 * 4294967279, 2147483659 * 2147483693):
        for c in [1, n - 1, n // 2] + [rng.randrange(n) for _ in range(3000)]:
            want = float(Fraction(c, n))
            want = 0.9999999999999999 if want >= 1.0 else want
            if L.or_unit_exact(c, n) != want:
                return False
    return True


def check_vector(L):
    # Eq. vectorize: Mv = 3 instances side by side equal their streams interleaved k-major
    ps = [2147483659, 2147483693, 4294967291]
    qs = [2147483693, 4294967279, 2147483659]
    es, N = [5, 7, 5], 40
    u64p = ctypes.POINTER(ctypes.c_uint64)
    arr = lambda xs: np.array(xs, np.uint64)
    p, q, e, a = arr(ps), arr(qs), arr(es), arr([A, A, A])
    m, s = arr([11, 22, 33]), arr([1, 1, 1])
    c = np.zeros(3 * N, np.uint64)
    if L.or_generate_vector(3, *(x.ctypes.data_as(u64p) for x in (p, q, e, a)), Q,
                            m.ctypes.data_as(u64p), s.ctypes.data_as(u64p), N,
                            c.ctypes.data_as(u64p), None) != 0:
        return False
    for g in range(3):
        rc, cg, _, _, _ = _gen(L, ps[g], qs[g], es[g], [11, 22, 33][g], 1, N)
        if rc != 0 or not (c[g::3] == cg).all():
            return False
    return True


def check_seek_parallel(L):
    # the skip sums split over threads (ranges started by jump-ahead) equal the serial walk
    p, q = 2147483659, 4294967291
    for a, s0, k in ((A, 7, 0), (A, 7, 1), (A, 7, 1000), (A, 99, 123457), (1, 99, 5000)):
        prm = P(p, q, 3, a, Q)
        out = []
        for fn in (L.or_seek, L.or_seek_parallel):
            m, s = ctypes.c_uint64(12345), ctypes.c_uint64(s0)
            if fn(ctypes.byref(prm), ctypes.byref(m), ctypes.byref(s), k) != 0:
                return False
            out.append((m.value, s.value))
        if out[0] != out[1]:
            return False
    return True


def check_unit_hard(L):
    # quotients next to midpoints between doubles (see division_cases)
    import division_cases as DC

    for k in (0, 3):
        p, q, _ = DC.EDGE_MODULI[k]
        n = p * q
        for c in DC.near_midpoint_ciphertexts(n, t_max=63, seed=k)[::7]:
            if L.or_unit(int(c), n) != DC.reference_unit(int(c), n):
                return False
    return True


def check_sample(L):
    # or_sample_many at 1-based indices equals the matching elements of or_generate
    u64p = ctypes.POINTER(ctypes.c_uint64)
    ptr = lambda x: x.ctypes.data_as(u64p)
    ps, qs, es, N = [2147483659, 4294967291], [2147483693, 4294967279], [5, 7], 3000
    ks_list = [np.array([1, 2, 3, 50, 51, 2999, 3000], np.uint64),
               np.array([1, 1000, 1001, 1500], np.uint64)]
    nk = np.array([len(k) for k in ks_list], np.uint64)
    koff = np.array([0, len(ks_list[0])], np.uint64)
    ks = np.concatenate(ks_list)
    m, s = np.array([11, 22], np.uint64), np.array([1, 1], np.uint64)
    c = np.zeros(len(ks), np.uint64)
    r = np.zeros(len(ks), np.float64)
    arr = lambda xs: np.array(xs, np.uint64)
    if L.or_sample_many(2, ptr(arr(ps)), ptr(arr(qs)), ptr(arr(es)), ptr(arr([A, A])), Q, ptr(m),
                        ptr(s), ptr(ks), ptr(koff), ptr(nk), ptr(c),
                        r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) != 0:
        return False
    for g in range(2):
        rc, cg, rg, _, _ = _gen(L, ps[g], qs[g], es[g], [11, 22][g], 1, N)
        idx = ks_list[g].astype(np.int64) - 1
        sl = slice(int(koff[g]), int(koff[g] + nk[g]))
        if rc != 0 or not (c[sl] == cg[idx]).all() or not (r[sl] == rg[idx]).all():
            return False
    return True


CHECKS = [check_primality, check_roots, check_skips, check_period_tiny_q, check_closed_form,
          check_rsa, check_unit, check_split, check_histogram, check_modes, check_unit_exact,
          check_vector, check_seek_parallel, check_unit_hard, check_sample]

MUTANTS = {
    "schrage_negative_branch": ("return (s1 >= s2) ? (s1 - s2) : (s1 + (Q - s2));",
                                "return (s1 >= s2) ? (s1 - s2) : (s1 + (Q - s2) - 1);"),
    "skip_wrong_modulus": ("return or_mulmod(a, s, Q);", "return or_mulmod(a, s, Q - 2);"),
    "message_before_skip": ("            s = s_direct;\n            m = or_addmod(m, s % n, n);\n            mp = (mp + s) % p;\n            mq = (mq + s) % q;",
                            "            m = or_addmod(m, s % n, n);\n            mp = (mp + s) % p;\n            mq = (mq + s) % q;\n            s = s_direct;"),
    "garner_no_reduction": ("uint64_t diff = (cp + p - (cq % p)) % p;",
                            "uint64_t diff = (cp + p - cq) % p;"),
    "guard_strict": ("double r = dc / dn;\n    if (r >= 1.0)\n        r = 0x1.fffffffffffffp-1;",
                     "double r = dc / dn;\n    if (r > 1.0)\n        r = 0x1.fffffffffffffp-1;"),
    "four_mr_bases": ("int bases = (n < ((uint64_t)1 << 32)) ? 5 : 12;",
                      "int bases = (n < ((uint64_t)1 << 32)) ? 4 : 12;"),
    "no_square": ("        b = or_mulmod(b, b, m);\n        e >>= 1;\n    }\n    return r;\n}\n\n/* b^e mod m for m < 2^32",
                  "        e >>= 1;\n    }\n    return r;\n}\n\n/* b^e mod m for m < 2^32"),
    "split_off_by_one": ("u128 k = (u128)gamma * (u128)((Q - 1) / Mv);",
                         "u128 k = (u128)(gamma + 1) * (u128)((Q - 1) / Mv);"),
    "division_by_reciprocal": ("double r = dc / dn;", "double r = dc * (1.0 / dn);"),
    "digit_rounded_product": ("return (uint64_t)(((u128)M * d) >> sh);",
                              "return (uint64_t)(r * (double)d);"),
    "tuple_digits_reversed": ("            bin += g * w;\n            w *= d;",
                              "            bin = bin * d + g;"),
    "q_exponent_from_p": ("uint64_t cq = or_powmod_native32(mq, eq, q);",
                          "uint64_t cq = or_powmod_native32(mq, ep, q);"),
    "unit_skip_rejected": ("a < 1 || a >= Q", "a < 2 || a >= Q"),
    "crt_exponent_wrong_modulus": ("return ra + a * t;", "return ra + b * t;"),
    "exact_division_truncates": ("    if (round_bit && (sticky || (m & 1)))\n        m++;\n", ""),
    "vector_substream_major": ("                c_out[k * Mv + g] = c;", "                c_out[g * N + k] = c;"),
    "sample_zero_based_index": ("int rc = or_seek(P, m_io, s_io, ks[j] - done);",
                                "int rc = or_seek(P, m_io, s_io, ks[j] - done - 1);"),
    "sample_position_not_kept": ("        done = ks[j];\n", "        done = ks[j] - 1;\n"),
    "parallel_seek_range_start": ("uint64_t s = or_mulmod(s0, or_powmod(a, lo, Q), Q);",
                                  "uint64_t s = or_mulmod(s0, or_powmod(a, lo + 1, Q), Q);"),
}


@pytest.fixture(scope="module")
def clean():
    return oracle.lib()


def test_pins_pass_on_the_oracle(clean):
    for chk in CHECKS:
        assert chk(clean), chk.__name__


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, name
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(before, after))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(so), str(mutated), "-lm"], check=True)
    L = oracle.load_library(str(so))
    failed = [chk.__name__ for chk in CHECKS if not chk(L)]
    assert failed, f"no pin catches the planted mistake {name}"
