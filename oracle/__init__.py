"""CPU oracle for the RSA-exponentiation generator (arXiv:1811.11629).

TEST INFRASTRUCTURE ONLY. The oracle is the plain, slow definition the GPU
library is checked against. Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and the oracle never imports the library.

The arithmetic lives in ``rsaprng_oracle.c`` (plain C, ``unsigned __int128``,
no GPU code). This module compiles it with gcc into ``_build/`` and wraps it
with ctypes. Each wrapper names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsaprng_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")

Q = (1 << 63) - 25  # skip modulus, Sec. V
ROUTE_CHECKED, ROUTE_PAPER, ROUTE_DIRECT = 0, 1, 2
E_SMALLEST, E_UNIFORM, E_AT_LEAST = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (OpenMP, no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """A ctypes handle with the oracle's signatures for the library at `path`."""
    L = ctypes.CDLL(path)
    _configure(L)
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _configure(L):
    u64, i32, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    pu64 = ctypes.POINTER(ctypes.c_uint64)
    pdbl = ctypes.POINTER(ctypes.c_double)
    sig = {
        "or_q_default": (u64, []),
        "or_mulmod": (u64, [u64, u64, u64]),
        "or_addmod": (u64, [u64, u64, u64]),
        "or_powmod": (u64, [u64, u64, u64]),
        "or_gcd": (u64, [u64, u64]),
        "or_invmod": (u64, [u64, u64]),
        "or_is_prime": (i32, [u64]),
        "or_count_primes": (None, [u64, u64, pu64, pu64]),
        "or_skip_next_direct": (u64, [u64, u64, u64]),
        "or_skip_next_schrage": (u64, [u64, u64, u64]),
        "or_skip_jump": (u64, [u64, u64, u64, u64]),
        "or_split_s0": (u64, [u64, u64, u64, u64, u64]),
        "or_encrypt_direct": (u64, [u64, u64, u64]),
        "or_crt_encrypt": (u64, [u64, u64, u64, u64, u64, u64]),
        "or_crt_encrypt2": (u64, [u64, u64, u64, u64, u64, u64, u64]),
        "or_crt_exponent": (u64, [u64, u64, u64, u64]),
        "or_unit": (dbl, [u64, u64]),
        "or_unit_exact": (dbl, [u64, u64]),
        "or_generate": (i32, [ctypes.c_void_p, pu64, pu64, u64, pu64, pdbl, i32]),
        "or_seek": (i32, [ctypes.c_void_p, pu64, pu64, u64]),
        "or_seek_parallel": (i32, [ctypes.c_void_p, pu64, pu64, u64]),
        "or_sample": (i32, [ctypes.c_void_p, pu64, pu64, pu64, u64, pu64, pdbl]),
        "or_sample_many": (i32, [u64, pu64, pu64, pu64, pu64, u64, pu64, pu64, pu64,
                                 pu64, pu64, pu64, pdbl]),
        "or_unit_many": (None, [pu64, u64, pdbl, u64]),
        "or_unit_exact_many": (None, [pu64, u64, pdbl, u64]),
        "or_generate_many": (i32, [u64, pu64, pu64, pu64, pu64, u64, pu64, pu64,
                                   pu64, pu64, pu64, pdbl, i32]),
        "or_max_threads": (i32, []),
        "or_generate_vector": (i32, [u64, pu64, pu64, pu64, pu64, u64, pu64, pu64, u64, pu64,
                                     pdbl]),
        "or_digit_of_unit": (u64, [dbl, u64]),
        "or_histogram": (i32, [ctypes.c_void_p, pu64, pu64, u64, u64, u64, i32, i32, pu64]),
        "or_histogram_many": (i32, [u64, pu64, pu64, pu64, pu64, u64, pu64, pu64, pu64, u64,
                                    u64, i32, i32, pu64]),
        "or_splitmix64_next": (u64, [pu64]),
        "or_params_from_seed": (i32, [u64, i32, u64, u64, pu64, pu64, pu64, pu64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _pd(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint64), ("q", ctypes.c_uint64), ("e", ctypes.c_uint64),
                ("a", ctypes.c_uint64), ("Q", ctypes.c_uint64), ("eq", ctypes.c_uint64)]


# --- thin wrappers (one per C function) ---------------------------------------------

def mulmod(a, b, m):
    return lib().or_mulmod(a, b, m)


def powmod(b, e, m):
    """b^e mod m by square-and-multiply (Sec. I)."""
    return lib().or_powmod(b, e, m)


def invmod(a, m):
    """a^{-1} mod m by extended Euclid (Eq. RSAd); 0 if not invertible."""
    return lib().or_invmod(a, m)


def gcd(a, b):
    return lib().or_gcd(a, b)


def is_prime(n: int) -> bool:
    """Trial division + deterministic Rabin-Miller (Sec. V)."""
    return bool(lib().or_is_prime(n))


def count_primes(lo: int, hi: int):
    """(#primes, #safe primes) in [lo, hi) using is_prime (Sec. V counts)."""
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    lib().or_count_primes(lo, hi, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def skip_next_direct(s, a, q=Q):
    """a s mod Q (Eq. congruentialgenerator1), 128-bit route."""
    return lib().or_skip_next_direct(s, a, q)


def skip_next_schrage(s, a, q=Q):
    """a s mod Q by steps WH1-WH3 of Eq. algorithm1."""
    return lib().or_skip_next_schrage(s, a, q)


def skip_jump(s0, a, k, q=Q):
    """s_0 a^k mod Q (Eq. pseudoskip)."""
    return lib().or_skip_jump(s0, a, k, q)


def split_s0(s0, a, mv, gamma, q=Q):
    """s_0 a^(gamma floor((Q-1)/Mv)) mod Q (Sec. VI)."""
    return lib().or_split_s0(s0, a, q, mv, gamma)


def encrypt_direct(m, e, n):
    """m^e mod n (Eq. encrypt)."""
    return lib().or_encrypt_direct(m, e, n)


def crt_encrypt(mp, mq, p, q, e, qinv_p):
    """CRT + Garner (Eq. CRTimplementation)."""
    return lib().or_crt_encrypt(mp, mq, p, q, e, qinv_p)


def unit(c, n) -> float:
    """r = c / n in IEEE doubles with the 1.0 guard (Eq. CodeFloatingPointStep)."""
    return lib().or_unit(c, n)


def splitmix64(state: int, count: int):
    """`count` SplitMix64 outputs from `state` (published definition)."""
    st = ctypes.c_uint64(state)
    return [lib().or_splitmix64_next(ctypes.byref(st)) for _ in range(count)]


def params_from_seed(seed: int, e_rule: int = E_SMALLEST, e_lo: int = 3, e_hi: int = 3):
    """(p, q, e, message seed) from one 64-bit seed; the rule is documented in the C file."""
    p, q, e, ms = (ctypes.c_uint64() for _ in range(4))
    rc = lib().or_params_from_seed(seed, e_rule, e_lo, e_hi, ctypes.byref(p), ctypes.byref(q),
                                   ctypes.byref(e), ctypes.byref(ms))
    if rc != 0:
        raise ValueError(f"or_params_from_seed failed ({rc})")
    return p.value, q.value, e.value, ms.value


def generate(p, q, e, m0, s0, count, a=2307085864, q_mod=Q, route=ROUTE_CHECKED, want_c=True,
             want_r=True, eq=0):
    """Outputs k = 1..count of one instance from state (m0, s0) (Eq. algorithm1).

    eq: exponent of the q residue (CRT exponents, Sec. V's note); 0 means eq = e.
    Returns (c, r, m_end, s_end); c is uint64, r float64 (None when not wanted).
    """
    P = _Params(p, q, e, a, q_mod, eq)
    m = ctypes.c_uint64(m0)
    s = ctypes.c_uint64(s0)
    c = np.empty(count, np.uint64) if want_c else None
    r = np.empty(count, np.float64) if want_r else None
    rc = lib().or_generate(ctypes.byref(P), ctypes.byref(m), ctypes.byref(s), count,
                           _p64(c) if c is not None else None,
                           _pd(r) if r is not None else None, route)
    if rc != 0:
        raise RuntimeError(f"oracle generate failed ({rc})")
    return c, r, m.value, s.value


def crt_exponent(p, q, ep, eq) -> int:
    """E = ep mod (p-1), E = eq mod (q-1), or 0 when no such E exists (Sec. V's note)."""
    return lib().or_crt_exponent(p, q, ep, eq)


def crt_encrypt2(mp, mq, p, q, ep, eq) -> int:
    """CRT(mp^ep mod p, mq^eq mod q) by Garner's formula."""
    return lib().or_crt_encrypt2(mp, mq, p, q, ep, eq, lib().or_invmod(q % p, p))


def seek(p, q, a, m0, s0, k, q_mod=Q):
    """State after k outputs from (m0, s0), without encryption (Sec. IV sums)."""
    P = _Params(p, q, 3, a, q_mod)
    m = ctypes.c_uint64(m0)
    s = ctypes.c_uint64(s0)
    rc = lib().or_seek(ctypes.byref(P), ctypes.byref(m), ctypes.byref(s), k)
    if rc != 0:
        raise RuntimeError(f"oracle seek failed ({rc})")
    return m.value, s.value


def seek_parallel(p, q, a, m0, s0, k, q_mod=Q):
    """seek over all host cores: the skip sum split into ranges started by jump-ahead."""
    P = _Params(p, q, 3, a, q_mod)
    m = ctypes.c_uint64(m0)
    s = ctypes.c_uint64(s0)
    rc = lib().or_seek_parallel(ctypes.byref(P), ctypes.byref(m), ctypes.byref(s), k)
    if rc != 0:
        raise RuntimeError(f"oracle seek_parallel failed ({rc})")
    return m.value, s.value


def sample_many(p, q, e, a, m, s, ks_list, q_mod=Q):
    """Sampled outputs of many instances; ks_list[i] = increasing 1-based indices.

    m, s (uint64 arrays) are advanced in place to each instance's last sample.
    Returns (c, r) concatenated in instance order.
    """
    p, q, e, a = (np.ascontiguousarray(x, dtype=np.uint64) for x in (p, q, e, a))
    nk = np.array([len(k) for k in ks_list], dtype=np.uint64)
    koff = np.zeros_like(nk)
    if len(nk) > 1:
        koff[1:] = np.cumsum(nk[:-1], dtype=np.uint64)
    ks = np.ascontiguousarray(np.concatenate([np.asarray(k, dtype=np.uint64) for k in ks_list])
                              if len(ks_list) else np.zeros(0, np.uint64))
    c = np.empty(len(ks), np.uint64)
    r = np.empty(len(ks), np.float64)
    rc = lib().or_sample_many(len(nk), _p64(p), _p64(q), _p64(e), _p64(a), q_mod, _p64(m),
                              _p64(s), _p64(ks), _p64(koff), _p64(nk), _p64(c), _pd(r))
    if rc != 0:
        raise RuntimeError(f"oracle sample_many failed ({rc})")
    return c, r


def unit_exact(c, n) -> float:
    """RN(c / n) of the exact rational, with the 1.0 guard (the other reading of the
    division of Eq. CodeFloatingPointStep)."""
    return lib().or_unit_exact(c, n)


def unit_exact_many(c: np.ndarray, n: int) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.uint64)
    r = np.empty(len(c), np.float64)
    lib().or_unit_exact_many(_p64(c), n, _pd(r), len(c))
    return r


def unit_many(c: np.ndarray, n: int) -> np.ndarray:
    """or_unit over an array (Eq. CodeFloatingPointStep)."""
    c = np.ascontiguousarray(c, dtype=np.uint64)
    r = np.empty(len(c), np.float64)
    lib().or_unit_many(_p64(c), n, _pd(r), len(c))
    return r


def generate_many(p, q, e, a, m, s, counts, offsets=None, route=ROUTE_CHECKED, want_c=True,
                  want_r=True, q_mod=Q):
    """Many instances at once (OpenMP over instances). m, s are advanced in place."""
    p, q, e, a = (np.ascontiguousarray(x, dtype=np.uint64) for x in (p, q, e, a))
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    if offsets is None:
        offsets = np.zeros_like(counts)
        if len(counts) > 1:
            offsets[1:] = np.cumsum(counts[:-1], dtype=np.uint64)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    total = int((offsets + counts).max()) if len(counts) else 0
    assert m.dtype == np.uint64 and s.dtype == np.uint64
    c = np.empty(total, np.uint64) if want_c else None
    r = np.empty(total, np.float64) if want_r else None
    rc = lib().or_generate_many(len(counts), _p64(p), _p64(q), _p64(e), _p64(a), q_mod, _p64(m),
                                _p64(s), _p64(counts), _p64(offsets),
                                _p64(c) if c is not None else None,
                                _pd(r) if r is not None else None, route)
    if rc != 0:
        raise RuntimeError(f"oracle generate_many failed ({rc})")
    return c, r


def digit_of_unit(r: float, d: int) -> int:
    """floor(r d), exactly, for a float output r in [0, 1) (Sec. VII's binning)."""
    return lib().or_digit_of_unit(r, d)


def histogram_many(p, q, e, a, m, s, counts, D, d, source=0, route=ROUTE_PAPER, q_mod=Q):
    """Frequency (D = 1) / serial (D > 1) test histogram (Sec. VII) of the next counts[i]
    outputs of each instance: non-overlapping D-tuples, bin = sum_i digit_i d^(i-1), digit
    floor(r d) (source 0) or c mod d (source 1). m, s are advanced in place."""
    p, q, e, a = (np.ascontiguousarray(x, dtype=np.uint64) for x in (p, q, e, a))
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    assert m.dtype == np.uint64 and s.dtype == np.uint64
    hist = np.zeros(int(d) ** int(D), np.uint64)
    rc = lib().or_histogram_many(len(counts), _p64(p), _p64(q), _p64(e), _p64(a), q_mod, _p64(m),
                                 _p64(s), _p64(counts), D, d, source, route, _p64(hist))
    if rc != 0:
        raise RuntimeError(f"oracle histogram_many failed ({rc})")
    return hist


def generate_vector(p, q, e, a, m, s, N, q_mod=Q):
    """The vectorised call of Sec. VI (Eq. vectorize): N steps of the Mv-vector update;
    returns (c, r) of length N * Mv in k-major order (element gamma of step k at
    k * Mv + gamma). m, s are advanced in place."""
    p, q, e, a = (np.ascontiguousarray(x, dtype=np.uint64) for x in (p, q, e, a))
    assert m.dtype == np.uint64 and s.dtype == np.uint64
    Mv = len(p)
    c = np.empty(N * Mv, np.uint64)
    r = np.empty(N * Mv, np.float64)
    rc = lib().or_generate_vector(Mv, _p64(p), _p64(q), _p64(e), _p64(a), q_mod, _p64(m), _p64(s),
                                  N, _p64(c), _pd(r))
    if rc != 0:
        raise RuntimeError(f"oracle generate_vector failed ({rc})")
    return c, r


def max_threads() -> int:
    return lib().or_max_threads()
