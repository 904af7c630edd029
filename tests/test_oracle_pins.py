"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests touches the GPU library. Each one checks the oracle
against something other than itself: printed constants (tests/golden/),
closed forms, invariants, brute force on tiny inputs, exact rational
arithmetic, or an independent library routine (sympy, Python big ints).
"""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
Q = GOLDEN["Q"]["value"]
ROOTS = [GOLDEN["default_root"]["value"]] + [
    a for a in GOLDEN["sezgin_roots"]["values"] if a not in GOLDEN["sezgin_not_primitive"]["values"]]
Q_MINUS_1_FACTORS = [2, 3, 17, 23, 319279, 456065899]  # distinct prime factors of Q-1


def test_q_value_and_largest_prime(oracle_mod):
    """Sec. V: Q = 2^63 - 25 is prime and no larger prime lies below 2^63."""
    O = oracle_mod
    assert Q == (1 << 63) - 25 == O.Q
    assert O.is_prime(Q)
    for x in range(Q + 1, 1 << 63):
        assert not O.is_prime(x)
    sympy = pytest.importorskip("sympy")
    assert sympy.prevprime(1 << 63) == Q


def test_q_minus_1_factorisation(oracle_mod):
    """Sec. V: Q-1 is coprime to all primes in [2^31, 2^32]; the factor list is complete."""
    O = oracle_mod
    exps = {2: 1, 3: 4, 17: 1, 23: 1, 319279: 1, 456065899: 1}
    prod = 1
    for f, k in exps.items():
        assert O.is_prime(f)
        prod *= f**k
    assert prod == Q - 1
    assert all(not ((1 << 31) <= f <= (1 << 32)) for f in exps)


def _is_primitive_root(O, a):
    if O.powmod(a, Q - 1, Q) != 1:
        return False
    return all(O.powmod(a, (Q - 1) // f, Q) != 1 for f in Q_MINUS_1_FACTORS)


def test_listed_roots_are_primitive(oracle_mod):
    """Notes to the skip generator: the recommended and Sezgin multipliers are primitive roots."""
    O = oracle_mod
    for a in ROOTS:
        assert _is_primitive_root(O, a), a


def test_listed_root_3163786287_is_a_quadratic_residue(oracle_mod):
    """Reading: one listed multiplier has a^((Q-1)/2) = 1, so it is not a primitive root."""
    O = oracle_mod
    a = 3163786287
    assert O.powmod(a, (Q - 1) // 2, Q) == 1
    assert not _is_primitive_root(O, a)


def test_smallest_primitive_roots(oracle_mod):
    """Sec. VII: 3, 6, 7, 10, 11 are the five smallest primitive roots mod Q."""
    O = oracle_mod
    found = [g for g in range(2, 12) if _is_primitive_root(O, g)]
    assert found == GOLDEN["smallest_roots"]["values"]


def test_restricted_roots_schrage_condition(oracle_mod):
    """Eq. restrictedprimitiveroots: 32-bit roots with q2 < q1, and WH1-WH3 equals a s mod Q."""
    O = oracle_mod
    rng = random.Random(7)
    for a in ROOTS + GOLDEN["smallest_roots"]["values"]:
        q1, q2 = Q // a, Q % a
        assert q2 < q1
        if a > 11:
            assert (1 << 31) <= a < (1 << 32)
        edge = [1, 2, Q - 1, Q - 2, q1 - 1, q1, q1 + 1, 2 * q1, (Q - 1) // 2]
        for s in edge + [rng.randrange(1, Q) for _ in range(2000)]:
            want = (a * s) % Q  # Python big integers
            assert O.skip_next_schrage(s, a) == want
            assert O.skip_next_direct(s, a) == want


def test_skip_jump_equals_iteration(oracle_mod):
    """Eq. congruentialgenerator1: s_k = a s_{k-1} mod Q = s_0 a^k mod Q."""
    O = oracle_mod
    for a in (ROOTS[0], ROOTS[3], 3):
        s0 = 123456789
        s = s0
        for k in range(1, 600):
            s = O.skip_next_schrage(s, a)
            if k % 37 == 0 or k < 5:
                assert O.skip_jump(s0, a, k) == s
        # a full-order element: a^(Q-1) = 1 returns the skip to s_0
        assert O.skip_jump(s0, a, Q - 1) == s0


def _sieve(lo, hi):
    """Primes in [lo, hi) by a segmented sieve of Eratosthenes (numpy)."""
    r = int(math.isqrt(hi)) + 1
    base = np.ones(r + 1, bool)
    base[:2] = False
    for i in range(2, int(math.isqrt(r)) + 1):
        if base[i]:
            base[i * i::i] = False
    small = np.nonzero(base)[0]
    seg = np.ones(hi - lo, bool)
    for pr in small:
        pr = int(pr)
        start = max(pr * pr, ((lo + pr - 1) // pr) * pr)
        seg[start - lo::pr] = False
    return lo + np.nonzero(seg)[0]


@pytest.mark.parametrize("lo", [1 << 31, (1 << 32) - (1 << 20), 3, 1 << 20])
def test_rabin_miller_matches_sieve(oracle_mod, lo):
    """Sec. V: bases {2,3,5,7,11} identify every prime below 2^32 (checked against a sieve)."""
    O = oracle_mod
    hi = lo + (1 << 20)
    primes = set(int(x) for x in _sieve(lo, hi))
    for x in range(lo | 1, hi, 2):
        assert O.is_prime(x) == (x in primes), x


def test_rabin_miller_rejects_strong_pseudoprimes(oracle_mod):
    """Sec. V: composites that fool the smaller base sets are still rejected."""
    O = oracle_mod
    # Smallest strong pseudoprimes to the first k prime bases (the sequence the paper cites).
    spsp = [2047, 1373653, 25326001, 3215031751, 2152302898747, 3474749660383,
            341550071728321, 3825123056546413051]
    sympy = pytest.importorskip("sympy")
    for x in spsp:
        assert not sympy.isprime(x)
        assert not O.is_prime(x)
    rng = random.Random(3)
    for _ in range(300):
        p = sympy.randprime(1 << 31, 1 << 32)
        q = sympy.randprime(1 << 31, 1 << 32)
        assert O.is_prime(p) and O.is_prime(q)
        assert not O.is_prime(p * q)
    for _ in range(300):
        x = rng.randrange(1 << 32, 1 << 64) | 1
        assert O.is_prime(x) == sympy.isprime(x)


@pytest.mark.slow
def test_prime_counts_sec5(oracle_mod):
    """Sec. V: 98,182,656 primes and 3,060,794 safe primes in [2^31, 2^32]."""
    n_primes, n_safe = oracle_mod.count_primes(1 << 31, 1 << 32)
    assert n_primes == GOLDEN["primes_2_31_2_32"]["value"]
    assert n_safe == GOLDEN["safe_primes_2_31_2_32"]["value"]


def _small_primes(lo, hi):
    return [x for x in range(lo, hi) if all(x % d for d in range(2, int(math.isqrt(x)) + 1))]


def test_encryption_is_a_permutation_tiny(oracle_mod):
    """Sec. III: m -> m^e mod n is a bijection of Z_n (brute force, tiny p, q); CRT = direct."""
    O = oracle_mod
    primes = _small_primes(3, 48)
    checked = 0
    for i, p in enumerate(primes):
        for q in primes[i + 1:]:
            n, phi = p * q, (p - 1) * (q - 1)
            qinv = pow(q, -1, p)
            for e in range(3, 24, 2):
                if math.gcd(e, phi) != 1:
                    continue
                img = [O.encrypt_direct(m, e, n) for m in range(n)]
                assert sorted(img) == list(range(n))
                for m in range(n):
                    assert O.crt_encrypt(m % p, m % q, p, q, e, qinv) == img[m]
                checked += 1
    assert checked > 100


def _random_instances(O, count, seed=11, e_rule=0, e_lo=3, e_hi=3):
    import workload

    seeds = workload.instance_seeds(seed, count)
    return [O.params_from_seed(int(s), e_rule, e_lo, e_hi) for s in seeds]


def test_rsa_round_trip_and_crt_residues(oracle_mod):
    """Eqs. decrypt/RSAd/decryptproof and CRTimplementation on 32-bit prime pairs."""
    O = oracle_mod
    rng = random.Random(5)
    for p, q, e, _ in _random_instances(O, 40, e_rule=1, e_lo=3, e_hi=65537):
        n = p * q
        lam = (p - 1) * (q - 1) // math.gcd(p - 1, q - 1)
        d_phi = pow(e, -1, (p - 1) * (q - 1))
        d_lam = pow(e, -1, lam)
        qinv = pow(q, -1, p)
        assert O.invmod(q % p, p) == qinv
        for m in [0, 1, 2, n - 1, n - 2] + [rng.randrange(n) for _ in range(50)]:
            c = O.encrypt_direct(m, e, n)
            assert O.powmod(c, d_phi, n) == m
            assert O.powmod(c, d_lam, n) == m
            assert c % p == pow(m % p, e, p)
            assert c % q == pow(m % q, e, q)
            cp, cq = c % p, c % q
            assert ((((cp - cq) * qinv) % p) * q + cq) == c  # Garner
            assert O.crt_encrypt(m % p, m % q, p, q, e, qinv) == c


def test_cribs_and_unit_exponent(oracle_mod):
    """Sec. IV cribs: 0, 1, n-1 map to themselves; Sec. VII: e = 1 gives c = m."""
    O = oracle_mod
    for p, q, e, _ in _random_instances(O, 20, seed=12):
        n = p * q
        for m in (0, 1, n - 1):
            assert O.encrypt_direct(m, e, n) == m
        c, _, _, _ = O.generate(p, q, 1, 17, 1, 50, route=O.ROUTE_CHECKED, want_r=False)
        # with e = 1 the outputs are the messages m_1.. themselves
        s, m = 1, 17
        msgs = []
        for _ in range(50):
            s = (ROOTS[0] * s) % Q
            m = (m + s) % n
            msgs.append(m)
        assert list(map(int, c)) == msgs


def _exact_unit(c, n):
    """RN(RN(c)/RN(n)) from exact rationals, then the 1.0 guard."""
    dc, dn = Fraction(float(c)), Fraction(float(n))
    r = float(dc / dn)  # correctly rounded quotient of the two doubles
    return 0.9999999999999999 if r >= 1.0 else r


def test_unit_conversion_exact_rounding(oracle_mod):
    """Eq. CodeFloatingPointStep and the r = 1.0 guard (Sec. V)."""
    O = oracle_mod
    rng = random.Random(9)
    assert 0.9999999999999999 == 1.0 - 2.0**-53
    differ = 0
    for p, q, _, _ in _random_instances(O, 30, seed=13):
        n = p * q
        assert n > 1 << 53
        cases = [0, 1, 2, n - 1, n - 2, n - 1024, n - 2048, n // 2, (1 << 53) - 1, 1 << 53,
                 (1 << 53) + 1]
        cases += [rng.randrange(n) for _ in range(400)]
        cases += [n - rng.randrange(1, 1 << 12) for _ in range(100)]
        for c in cases:
            r = O.unit(c, n)
            assert r == _exact_unit(c, n)
            assert 0.0 <= r < 1.0
            if r != float(Fraction(c, n)):
                differ += 1
        assert O.unit(n - 1, n) == 1.0 - 2.0**-53
        assert O.unit(0, n) == 0.0
    # Double rounding makes the reading matter: RN(RN(c)/RN(n)) != RN(c/n) for many draws.
    assert differ > 100


def test_unit_near_midpoints(oracle_mod):
    """Eq. CodeFloatingPointStep at its hardest inputs: RN(c)/RN(n) next to a midpoint.

    The oracle's (double)c / (double)n must equal Python's correctly rounded
    integer division of the two correctly rounded conversions on ciphertexts
    built to put the quotient within 2^-106 .. 2^-90 relative of a midpoint
    between neighbouring doubles, for moduli at the edges of the range.
    """
    import division_cases as DC

    O = oracle_mod
    for k, (p, q, _) in enumerate(DC.EDGE_MODULI):
        n = p * q
        c = DC.near_midpoint_ciphertexts(n, seed=k)
        assert len(c) >= 100000
        want = np.array([DC.reference_unit(int(x), n) for x in c])
        got = O.unit_many(c, n)
        bad = np.nonzero(got.view(np.uint64) != want.view(np.uint64))[0]
        assert len(bad) == 0, (n, c[bad[:3]])
        # the construction really lands next to midpoints (odd significands of RN(n))
        if DC.split_double(float(n))[0] & 1:
            d = [DC.midpoint_distance_ulps(int(x), n) for x in c[::max(1, len(c) // 400)]]
            assert np.mean(np.array(d) < 2.0**-40) > 0.75


def test_sample_many_matches_generate(oracle_mod):
    """The sampler behind every full-size check: output k (1-based) of or_sample_many is
    element k - 1 of or_generate, and each instance ends at its last sampled output."""
    O = oracle_mod
    rng = np.random.default_rng(31)
    inst = _random_instances(O, 5, seed=41, e_rule=1, e_lo=3, e_hi=65537)
    N = 100000
    ks_list, full = [], []
    for j, (p, q, e, ms) in enumerate(inst):
        n = p * q
        c, r, m_end, s_end = O.generate(p, q, e, ms % n, 1, N, route=O.ROUTE_DIRECT)
        pick = {1, 2, N} | set(int(x) for x in rng.integers(1, N + 1, 40)) | {777, 778, 779}
        ks = np.array(sorted(pick)[: 10 + 8 * j], dtype=np.uint64)
        ks_list.append(ks)
        full.append((c, r))
    arr = lambda i: np.array([x[i] for x in inst], dtype=np.uint64)
    m = np.array([ms % (p * q) for p, q, _, ms in inst], dtype=np.uint64)
    s = np.ones(len(inst), np.uint64)
    a = np.full(len(inst), ROOTS[0], np.uint64)
    c_s, r_s = O.sample_many(arr(0), arr(1), arr(2), a, m, s, ks_list)
    off = 0
    for j, (p, q, e, ms) in enumerate(inst):
        ks = ks_list[j].astype(np.int64)
        c, r = full[j]
        assert (c_s[off:off + len(ks)] == c[ks - 1]).all()
        assert (r_s[off:off + len(ks)].view(np.uint64) == r[ks - 1].view(np.uint64)).all()
        off += len(ks)
        _, _, m_last, s_last = O.generate(p, q, e, ms % (p * q), 1, int(ks[-1]),
                                          route=O.ROUTE_DIRECT, want_c=False, want_r=False)
        assert (int(m[j]), int(s[j])) == (m_last, s_last)


def test_tiny_q_period_and_message_counts(oracle_mod):
    """Sec. IV: with a primitive root a mod Q' and gcd(Q'(Q'-1)/2, n) = 1 the period is
    (Q'-1) n and every message appears exactly Q'-1 times per period."""
    O = oracle_mod
    qp, a = 47, 5
    assert sorted(pow(a, k, qp) for k in range(1, qp)) == list(range(1, qp))  # primitive
    p, q, e = 5, 11, 3
    n = p * q
    b = qp * (qp - 1) // 2
    assert math.gcd(b, n) == 1
    period = (qp - 1) * n
    m0, s0 = 7, 1
    msgs, _, m_end, s_end = O.generate(p, q, 1, m0, s0, 2 * period + 5, a=a, q_mod=qp,
                                       route=O.ROUTE_CHECKED, want_r=False)
    msgs = [int(x) for x in msgs]
    # the state first returns after exactly (Q'-1) n steps
    state = [(m0, s0)]
    s, m = s0, m0
    for k in range(1, period + 1):
        s = O.skip_next_schrage(s, a, qp)
        m = msgs[k - 1]
        state.append((m, s))
    assert state[period] == state[0]
    assert all(state[k] != state[0] for k in range(1, period))
    counts = np.bincount(np.array(msgs[:period]), minlength=n)
    assert (counts == qp - 1).all()
    # m_{k+Q'-1} = m_k + Q'(Q'-1)/2 mod n
    for k in range(0, period):
        assert msgs[k + qp - 1] == (msgs[k] + b) % n
    # and the ciphertexts of the same sequence with e = 3 are their encryptions
    cs, _, _, _ = O.generate(p, q, e, m0, s0, period, a=a, q_mod=qp, route=O.ROUTE_CHECKED,
                             want_r=False)
    assert [int(x) for x in cs] == [pow(m, e, n) for m in msgs[:period]]


def test_closed_form_pseudoskip(oracle_mod):
    """Eq. pseudoskip: for k = u(Q'-1) + v, m_k = m_0 + u b + sum_{j=1..v} a^(v_0+j) mod Q'."""
    O = oracle_mod
    qp, a, v0 = 47, 5, 9
    p, q = 5, 11
    n = p * q
    b = (qp * (qp - 1) // 2) % n
    s0 = pow(a, v0, qp)
    m0 = 3
    msgs, _, _, _ = O.generate(p, q, 1, m0, s0, 5 * (qp - 1) + 20, a=a, q_mod=qp,
                               route=O.ROUTE_CHECKED, want_r=False)
    for k in range(1, len(msgs) + 1):
        u, v = divmod(k, qp - 1)
        closed = (m0 + u * b + sum(pow(a, v0 + j, qp) for j in range(1, v + 1))) % n
        assert int(msgs[k - 1]) == closed, k


def test_closed_form_full_q(oracle_mod):
    """Eq. pseudoskip at the real Q: m_k = m_0 + sum_{j=1..k} (s_0 a^j mod Q) mod n."""
    O = oracle_mod
    p, q, e, ms = _random_instances(O, 1, seed=21)[0]
    n = p * q
    m0, s0 = ms % n, 1
    cs, rs, m_end, s_end = O.generate(p, q, e, m0, s0, 300, route=O.ROUTE_CHECKED)
    acc = m0
    for k in range(1, 301):
        acc = (acc + pow(ROOTS[0], k, Q) * s0 % Q) % n
        assert int(cs[k - 1]) == pow(acc, e, n)
        assert float(rs[k - 1]) == _exact_unit(pow(acc, e, n), n)
    assert m_end == acc and s_end == pow(ROOTS[0], 300, Q)


def test_routes_agree_long(oracle_mod):
    """Eq. algorithm1 (CRT + Schrage) and the 128-bit route give identical streams."""
    O = oracle_mod
    for p, q, e, ms in _random_instances(O, 6, seed=22, e_rule=1, e_lo=3, e_hi=65537):
        n = p * q
        c1, r1, m1, s1 = O.generate(p, q, e, ms % n, 1, 20000, route=O.ROUTE_PAPER)
        c2, r2, m2, s2 = O.generate(p, q, e, ms % n, 1, 20000, route=O.ROUTE_DIRECT)
        assert (c1 == c2).all() and (r1 == r2).all() and (m1, s1) == (m2, s2)
        O.generate(p, q, e, ms % n, 1, 5000, route=O.ROUTE_CHECKED)


def test_split_substreams(oracle_mod):
    """Sec. VI: substream gamma starts at s_0 a^(gamma floor((Q-1)/Mv)) and is the parent's
    skip sequence shifted by that many steps (checked in full on a tiny Q')."""
    O = oracle_mod
    s0, a = 1, ROOTS[0]
    for mv in (1, 2, 32, 1000):
        for g in (0, 1, mv - 1):
            assert O.split_s0(s0, a, mv, g) == pow(a, g * ((Q - 1) // mv), Q)
    qp, a2 = 47, 5
    for mv in (2, 23, 46):
        stride = (qp - 1) // mv
        seq = [1]
        for _ in range(qp - 1):
            seq.append(O.skip_next_direct(seq[-1], a2, qp))
        for g in range(mv):
            assert O.split_s0(1, a2, mv, g, q=qp) == seq[g * stride]
    vals = {O.split_s0(1, a2, 46, g, q=qp) for g in range(46)}
    assert len(vals) == 46  # all substreams start at distinct skips


def test_splitmix64_published_value_and_numpy_twin(oracle_mod):
    """The input generator: SplitMix64 from state 0 (reference value) and the numpy twin."""
    import workload

    O = oracle_mod
    assert O.splitmix64(0, 1)[0] == int(GOLDEN["splitmix64_seed0_first"]["value"], 16)
    for st in (0, 1, 2**63 + 5, 12345):
        assert O.splitmix64(st, 20) == [int(x) for x in workload.splitmix64(st, 20)]


def test_params_from_seed_rules(oracle_mod):
    """Instance parameters: 32-bit primes with the top bit set, p != q, the exponent rules."""
    O = oracle_mod
    sympy = pytest.importorskip("sympy")
    import workload

    for rule, lo, hi in ((0, 3, 3), (1, 3, 65537), (1, 3, 257), (2, 3, 3), (2, 17, 17)):
        for s in workload.instance_seeds(99 + rule, 25):
            p, q, e, ms = O.params_from_seed(int(s), rule, lo, hi)
            assert p != q and sympy.isprime(p) and sympy.isprime(q)
            assert (1 << 31) <= p < (1 << 32) and (1 << 31) <= q < (1 << 32)
            phi = (p - 1) * (q - 1)
            assert e % 2 == 1 and math.gcd(e, phi) == 1
            if rule in (0, 2):
                start = 3 if rule == 0 else lo
                assert e >= start and all(math.gcd(x, phi) != 1 for x in range(start, e, 2))
            else:
                assert lo <= e <= hi
    # the first prime candidate is the first SplitMix64 draw that is prime
    st = 77
    draws = O.splitmix64(st, 64)
    cands = [(x >> 32) | 0x80000001 for x in draws]
    p, q, _, _ = O.params_from_seed(st)
    first = [c for c in cands if sympy.isprime(c)]
    assert p == first[0] and q == [c for c in first[1:] if c != p][0]


def test_period_claim_sec5():
    """Sec. V / abstract: P = (Q-1) n ~ 2^126 ~ 8.5e37 for n close to Q."""
    assert abs((Q - 1) * Q / GOLDEN["period_lower_bound"]["value"] - 1) < 0.001
    assert abs((Q - 1) * Q / 2.0**126 - 1) < 1e-15
