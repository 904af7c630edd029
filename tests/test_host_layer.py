"""Host-side checks that need no GPU: the library loads and exports its ABI,
and its host parameter layer agrees with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "rsaprng.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsaprng_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def R():
    import paper_1811_11629_gb300 as R

    R._lib.load()
    return R


def test_library_exports_every_declared_symbol(R):
    L = R._lib.load()
    declared = _declared_symbols()
    assert len(declared) >= 40
    for name in declared:
        assert hasattr(L, name), name
    # and the binding covers the same set
    assert set(declared) == set(R._lib.SIGNATURES), set(declared) ^ set(R._lib.SIGNATURES)


def test_strerror_covers_codes(R):
    L = R._lib.load()
    for code in list(R._lib.ERRORS) + [0]:
        msg = L.rsaprng_strerror(code).decode()
        assert msg and msg != "unknown error"


def test_is_prime_matches_oracle(R, oracle_mod):
    rng = np.random.default_rng(1)
    xs = list(rng.integers(1 << 31, 1 << 32, 20000, dtype=np.uint64))
    xs += list(rng.integers(1, 1 << 63, 2000, dtype=np.uint64))
    xs += [2, 3, 4, 2047, 3215031751, 2152302898747, 3825123056546413051, (1 << 63) - 25,
           (1 << 61) - 1, (1 << 64) - 59]
    for x in xs:
        assert R.is_prime(int(x)) == oracle_mod.is_prime(int(x)), int(x)


@pytest.mark.parametrize("rule,lo,hi", [(0, 3, 3), (1, 3, 65537), (1, 3, 257), (2, 3, 3),
                                        (2, 65537, 65537)])
def test_params_from_seed_matches_oracle(R, oracle_mod, rule, lo, hi):
    for s in workload.instance_seeds(1234 + rule, 300):
        assert R.params_from_seed(int(s), rule, lo, hi) == \
            oracle_mod.params_from_seed(int(s), rule, lo, hi)


def test_allowed_roots(R):
    listed = [2307085864, 3157107955, 3200261722, 3211103532, 3338736601, 3423977237,
              3465965455, 3474009732, 3512424704, 3, 6, 7, 10, 11]
    for a in listed:
        assert R.root_allowed(a)
    assert R.root_allowed(1)  # the unit / constant skip of Sec. IV
    for a in [3163786287, 2, 4, 5, 12, 2307085865, 0]:
        assert not R.root_allowed(a)


def test_parameter_validation_codes(R):
    """Fault injection on the host: bad primes, ranges, equal primes, bad exponents."""
    C = R._lib.CODES
    p, q = 4294967291, 4294967279  # the two largest primes below 2^32
    assert R.validate_params(p, q, 3) in (0, C["ERR_E"])
    e_ok = next(e for e in range(3, 200, 2) if math.gcd(e, (p - 1) * (q - 1)) == 1)
    assert R.validate_params(p, q, e_ok) == 0
    assert R.validate_params(p, p, e_ok) == C["ERR_P_EQ_Q"]
    assert R.validate_params(p, 4294967295, e_ok) == C["ERR_NOT_PRIME"]
    assert R.validate_params(p, 65521, e_ok) == C["ERR_RANGE"]
    assert R.validate_params(1 << 32, q, e_ok) == C["ERR_RANGE"]
    assert R.validate_params(p, q, e_ok + 1) == C["ERR_E"]
    assert R.validate_params(p, q, 1) == C["ERR_E"]
    bad_e = next(e for e in range(3, 2000, 2) if math.gcd(e, (p - 1) * (q - 1)) != 1)
    assert R.validate_params(p, q, bad_e) == C["ERR_E"]
    # a prime whose (p-1)/2 is composite fails the safe-prime rule of Sec. V
    assert not R.is_prime((p - 1) // 2) or not R.is_prime((q - 1) // 2)
    assert R.validate_params(p, q, e_ok, require_safe=True) == C["ERR_NOT_PRIME"]


def test_chi2_uniform_host_helper(R):
    """rsaprng_chi2_uniform against the chi^2 sum written out with numpy."""
    rng = np.random.default_rng(3)
    h = rng.integers(0, 50, 4096).astype(np.uint64)
    chi2, total = R.chi2_uniform(h)
    E = h.sum() / len(h)
    want = float(((h.astype(np.float64) - E) ** 2 / E).sum())
    assert total == int(h.sum())
    assert abs(chi2 - want) <= 1e-9 * max(1.0, want)
    flat = np.full(64, 9, np.uint64)
    assert R.chi2_uniform(flat) == (0.0, 576)
    with pytest.raises(R.RsaPrngError):
        R.chi2_uniform(np.zeros(8, np.uint64))


def test_autotune_cache_file_round_trip(R, tmp_path):
    """The tuning cache's text file (no GPU needed): entries load, save back line for
    line, and a malformed file is refused without touching the entries held."""
    L = R._lib.load()
    L.rsaprng_autotune_cache_clear()
    lines = ["sm103-x152/req2^10-mean2^14-max2^23/rounding0/e6 modexp=1 divide=4 threads=128 "
             "numbers=16 blocks_per_sm=0 chunk=262144 streams_per_block=2 unroll=8 pieces_per_block=1 "
             "rounding=0",
             "sm103-x152/req2^0-mean2^19-max2^19/rounding0/e4 modexp=1 divide=3 threads=256 "
             "numbers=8 blocks_per_sm=4 chunk=65536 streams_per_block=1 unroll=0 pieces_per_block=4 "
             "rounding=0"]
    src = tmp_path / "in.txt"
    src.write_text("\n".join(lines) + "\n")
    assert L.rsaprng_autotune_cache_load(str(src).encode()) == 0
    assert L.rsaprng_autotune_cache_size() == 2
    out = tmp_path / "out.txt"
    assert L.rsaprng_autotune_cache_save(str(out).encode()) == 0
    assert sorted(out.read_text().splitlines()) == sorted(lines)
    bad = tmp_path / "bad.txt"
    bad.write_text("key modexp=1 divide=oops\n")
    assert L.rsaprng_autotune_cache_load(str(bad).encode()) == R._lib.CODES["ERR_ARG"]
    assert L.rsaprng_autotune_cache_load(str(tmp_path / "missing").encode()) == \
        R._lib.CODES["ERR_ARG"]
    assert L.rsaprng_autotune_cache_size() == 2
    L.rsaprng_autotune_cache_clear()
    assert L.rsaprng_autotune_cache_size() == 0


def _latency_shape(R, n, sms, exact):
    L = R._lib.load()
    T, per = ctypes.c_int32(), ctypes.c_int32()
    assert L.rsaprng_latency_shape(n, sms, int(exact), ctypes.byref(T), ctypes.byref(per)) == 0
    return T.value, per.value


def test_latency_shape_rule(R):
    """The single-launch plain call's tile for draws that fit one wave of 512 x 16
    tiles: whole warps, 128 to 512 threads, 12-16 outputs per thread, at most one
    tile per SM, and of those the least per-scheduler work plus chain length,
    L (max(ceil(T / 128), 2) + 1), smaller L on a tie (checked against every
    admissible shape)."""
    for sms in (148, 152, 160):
        for n in (1, 1000, 8191, 8192, 100_000, 300_000, 600_000, 800_000, 1_000_000,
                  1_100_000, 8192 * sms - 1, 8192 * sms):
            for exact in (False, True):
                T, L = _latency_shape(R, n, sms, exact)
                assert T % 32 == 0 and 128 <= T <= 512
                assert L == 16 if exact else L in (12, 13, 14, 16)
                assert -(-n // (T * L)) <= sms  # at most one tile per SM
                cost = lambda t, l: l * (max(-(-t // 128), 2) + 1)
                for l2 in ((16,) if exact else (12, 13, 14, 16)):
                    for t2 in range(128, 513, 32):
                        if -(-n // (t2 * l2)) <= sms:
                            assert (cost(T, L), L) <= (cost(t2, l2), l2), (n, sms, T, L, t2, l2)
                # the fewest threads for that L that still keep one tile per SM
                assert T == 128 or -(-n // ((T - 32) * L)) > sms
    # the shapes measured on 152 SMs
    assert _latency_shape(R, 1_000_000, 152, False) == (512, 13)
    assert _latency_shape(R, 800_000, 152, False) == (384, 14)
    assert _latency_shape(R, 300_000, 152, False) == (192, 12)
    # a draw no shape covers on one tile per SM (up to the largest count) gets 512 x 16
    assert _latency_shape(R, 2**64 - 1, 152, False) == (512, 16)
    assert _latency_shape(R, 8192 * 152 + 1, 152, True) == (512, 16)
    L = R._lib.load()
    x = ctypes.c_int32()
    assert L.rsaprng_latency_shape(10, 0, 0, ctypes.byref(x), ctypes.byref(x)) != 0
    assert L.rsaprng_latency_shape(10, 152, 0, None, ctypes.byref(x)) != 0
