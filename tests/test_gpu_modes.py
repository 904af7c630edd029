"""GPU parity of the generator's modes against the oracle:

- the unit and constant skips of Sec. IV (multiplier a = 1),
- CRT exponents (the p and q residues raised to different exponents, the
  note on large exponents in Sec. V),
- the exact-rational reading of the division, r = RN(c / n).
All comparisons are bit-exact.
"""
import math

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1811_11629_gb300 as R  # noqa: E402

A = R.DEFAULT_ROOT
TILES = [(R.MODEXP_CRT32, R.DIVIDE_RECIP, 128, 16), (R.MODEXP_CRT32, R.DIVIDE_INT, 256, 8),
         (R.MODEXP_CRT32, R.DIVIDE_HYBRID, 64, 4), (R.MODEXP_MONT64, R.DIVIDE_FP64, 512, 2),
         (R.MODEXP_MONT64, R.DIVIDE_RECIP, 128, 8)]


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def pq(O, seed):
    p, q, e, ms = O.params_from_seed(int(workload.instance_seeds(seed, 1)[0]))
    return p, q, e, ms % (p * q)


def run(ctx, ids, N):
    c = torch.empty(len(ids) * N, dtype=torch.int64, device="cuda")
    r = torch.empty(len(ids) * N, dtype=torch.float64, device="cuda")
    ctx.generate_batch(ids, np.full(len(ids), N, np.uint64), out_r=r, out_c=c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64).reshape(len(ids), N), r.cpu().numpy().reshape(len(ids), N)


def check(O, got_c, got_r, p, q, e, m0, s0, a=A, eq=0, exact=False):
    N = len(got_c)
    c, r, m1, s1 = O.generate(p, q, e, m0, s0, N, a=a, eq=eq)
    np.testing.assert_array_equal(got_c, c)
    want_r = O.unit_exact_many(c, p * q) if exact else r
    bad = np.nonzero(bits(got_r) != bits(want_r))[0]
    assert len(bad) == 0, f"r mismatch at {bad[:5]}"
    return m1, s1


@pytest.mark.parametrize("modexp,divide,T,L", TILES)
def test_unit_and_constant_skip(O, modexp, divide, T, L):
    ctx = R.Context(8, modexp=modexp, divide=divide, threads_per_block=T, numbers_per_thread=L)
    rng = np.random.default_rng(21)
    inst = []
    for k, seed in enumerate((31, 32, 33)):
        p, q, e, m0 = pq(O, seed)
        b = 1 if k == 0 else int(rng.integers(2, (1 << 63) - 25))
        inst.append((ctx.create_ex(p, q, e, 1, m0, b), p, q, e, m0, b))
    ids = np.array([x[0] for x in inst], np.uint32)
    N = 50021
    gc, gr = run(ctx, ids, N)
    for j, (i, p, q, e, m0, b) in enumerate(inst):
        m1, s1 = check(O, gc[j], gr[j], p, q, e, m0, b, a=1)
        assert ctx.get_state(int(i)) == (m1, s1)
        assert s1 == b  # the skip never changes
        n = p * q
        assert int(gc[j][9]) == pow((m0 + 10 * b) % n, e, n)
    with pytest.raises(R.RsaPrngError):
        ctx.split(int(ids[0]), 4)


def test_constant_skip_long_stream_in_pieces(O):
    """A long constant-skip stream is cut into pieces; the skip-sum pass runs with a = 1."""
    ctx = R.Context(4, chunk=1 << 16)
    p, q, e, m0 = pq(O, 34)
    b = 987654321987654321
    i = ctx.create_ex(p, q, e, 1, m0, b)
    N = 2_000_003
    r = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.generate_f64(i, N, r)
    torch.cuda.synchronize()
    _, want, m1, s1 = O.generate(p, q, e, m0, b, N, a=1, want_c=False)
    assert (bits(r.cpu().numpy()) == bits(want)).all()
    assert ctx.get_state(i) == (m1, s1) == ((m0 + N * b) % (p * q), b)


def crt_pairs(O, seeds):
    """(p, q, e_p, e_q, m0) with e_p != e_q, both with and without a single exponent."""
    out = []
    for seed in seeds:
        p, q, _, m0 = pq(O, seed)
        ep = next(x for x in range(5, 300, 2) if math.gcd(x, p - 1) == 1)
        eqs = [x for x in range(3, 600, 2) if x != ep and math.gcd(x, q - 1) == 1]
        consistent = [x for x in eqs if O.crt_exponent(p, q, ep, x)]
        other = [x for x in eqs if not O.crt_exponent(p, q, ep, x)]
        for eq in (consistent[:1] + other[:1]):
            out.append((p, q, ep, eq, m0))
    return out


@pytest.mark.parametrize("divide,T,L", [(R.DIVIDE_RECIP, 128, 16), (R.DIVIDE_INT, 256, 8),
                                        (R.DIVIDE_HYBRID, 64, 2)])
def test_crt_exponents(O, divide, T, L):
    ctx = R.Context(16, divide=divide, threads_per_block=T, numbers_per_thread=L)
    pairs = crt_pairs(O, range(41, 47))
    assert any(O.crt_exponent(p, q, ep, eq) == 0 for p, q, ep, eq, _ in pairs)
    assert any(O.crt_exponent(p, q, ep, eq) != 0 for p, q, ep, eq, _ in pairs)
    ids = np.array([ctx.create_crt(p, q, ep, eq, A, m0, 1) for p, q, ep, eq, m0 in pairs],
                   np.uint32)
    for i, (p, q, ep, eq, m0) in zip(ids, pairs):
        assert ctx.exponents(int(i)) == (ep, eq)
    N = 30011
    gc, gr = run(ctx, ids, N)
    for j, (p, q, ep, eq, m0) in enumerate(pairs):
        m1, s1 = check(O, gc[j], gr[j], p, q, ep, m0, 1, eq=eq)
        assert ctx.get_state(int(ids[j])) == (m1, s1)


def test_crt_exponents_refused_by_the_64_bit_route(O):
    ctx = R.Context(4, modexp=R.MODEXP_MONT64)
    (p, q, ep, eq, m0), = crt_pairs(O, [48])[:1]
    i = ctx.create_crt(p, q, ep, eq, A, m0, 1)
    r = torch.empty(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RsaPrngError):
        ctx.generate_f64(i, 1000, r)
    assert ctx.get_state(i) == (m0, 1)
    # the autotuner leaves the 64-bit route out for such instances
    tuned = ctx.autotune([i], [100000], reps=1)
    assert tuned["modexp"] == R.MODEXP_CRT32


@pytest.mark.parametrize("modexp,divide,T,L", TILES)
def test_exact_rational_division(O, modexp, divide, T, L):
    ctx = R.Context(8, modexp=modexp, divide=divide, threads_per_block=T, numbers_per_thread=L,
                    rounding=R._lib.ROUND_EXACT)
    seeds = workload.instance_seeds(51, 3)
    first = ctx.create_seeded(seeds, R.E_UNIFORM, 3, 257)
    ids = np.arange(first, first + 3, dtype=np.uint32)
    N = 40009
    gc, gr = run(ctx, ids, N)
    for j, s in enumerate(seeds):
        p, q, e, ms = O.params_from_seed(int(s), R.E_UNIFORM, 3, 257)
        check(O, gc[j], gr[j], p, q, e, ms % (p * q), 1, exact=True)


def test_exact_rational_unit_step_edges(O):
    """rsaprng_unit_f64 under the exact reading, on random, tiny, near-n and near-tie c."""
    ctx = R.Context(4, rounding=R._lib.ROUND_EXACT)
    p, q, e, m0 = pq(O, 52)
    i = ctx.create(p, q, e, m0)
    n = p * q
    rng = np.random.default_rng(5)
    c = np.concatenate([rng.integers(0, n, 200000, dtype=np.uint64),
                        rng.integers(1, 1 << 12, 2000, dtype=np.uint64),
                        np.uint64(n) - rng.integers(1, 1 << 14, 2000, dtype=np.uint64),
                        np.array([0, 1, 2, n - 1, n - 2, n >> 1, n // 3], np.uint64)])
    # c/n next to the midpoint of two neighbouring doubles
    from fractions import Fraction
    ties = []
    for x in rng.random(3000):
        mid = (Fraction(float(x)) + Fraction(math.nextafter(float(x), 1.0))) / 2
        t = math.floor(mid * n)
        ties += [t, t + 1]
    c = np.concatenate([c, np.array([t for t in ties if t < n], np.uint64)])
    dc = torch.from_numpy(c.view(np.int64)).cuda()
    dr = torch.empty(len(c), dtype=torch.float64, device="cuda")
    assert ctx.L.rsaprng_unit_f64(ctx.h, i, len(c), dc.data_ptr(), dr.data_ptr(), 0,
                                  torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    want = O.unit_exact_many(c, n)
    got = dr.cpu().numpy()
    bad = np.nonzero(bits(got) != bits(want))[0]
    assert len(bad) == 0, f"c={c[bad[:3]]}"


def test_modes_through_the_histogram_consumer(O):
    """Constant skip and CRT exponents through the fused histogram consumer."""
    ctx = R.Context(8)
    p, q, e, m0 = pq(O, 53)
    i1 = ctx.create_ex(p, q, e, 1, m0, 12345)
    (p2, q2, ep, eq, m2), = crt_pairs(O, [54])[:1]
    i2 = ctx.create_crt(p2, q2, ep, eq, A, m2, 1)
    counts = [100003, 77777]
    hist = ctx.histogram([i1, i2], counts, 2, 64, R.HIST_HIGH)
    torch.cuda.synchronize()
    want = np.zeros(64 * 64, np.uint64)
    for (pp, qq, ee, mm, ss, aa, eqq), N in zip([(p, q, e, m0, 12345, 1, 0),
                                                 (p2, q2, ep, m2, 1, A, eq)], counts):
        _, r, _, _ = O.generate(pp, qq, ee, mm, ss, N, a=aa, eq=eqq)
        d = (r * 64).astype(np.int64)
        t = N // 2
        np.add.at(want, d[0:2 * t:2] + 64 * d[1:2 * t:2], 1)
    np.testing.assert_array_equal(hist.cpu().numpy().view(np.uint64), want)
