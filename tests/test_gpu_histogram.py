"""GPU parity of the fused histogram consumer (Sec. VII's one-dimensional
frequency test and D-dimensional serial test): rsaprng_histogram against the
oracle's histogram of the same outputs. Counts are integers, so the bar is
equality; the instance states after the call must match as well.
"""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1811_11629_gb300 as R  # noqa: E402

A = R.DEFAULT_ROOT
HIGH, LOW = R.HIST_HIGH, R.HIST_LOW


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def seeded(ctx, O, master, k, rule, lo, hi):
    seeds = workload.instance_seeds(master, k)
    first = ctx.create_seeded(seeds, rule, lo, hi)
    ids = np.arange(first, first + k, dtype=np.uint32)
    par = [O.params_from_seed(int(s), rule, lo, hi) for s in seeds]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    m0 = np.array([int(x[3]) % (int(x[0]) * int(x[1])) for x in par], np.uint64)
    return ids, p, q, e, m0


def oracle_hist(O, p, q, e, m, s, counts, D, d, source):
    """The oracle's histogram; m, s (copies) are advanced and returned."""
    m, s = m.copy(), s.copy()
    a = np.full(len(p), A, np.uint64)
    h = O.histogram_many(p, q, e, a, m, s, np.asarray(counts, np.uint64), D, d, source)
    return h, m, s


def host(hist):
    torch.cuda.synchronize()
    return hist.cpu().numpy().view(np.uint64)


CASES = [(1, 1 << 20, HIGH), (1, 1000, HIGH), (2, 1024, HIGH), (3, 100, HIGH), (5, 16, HIGH),
         (6, 10, HIGH), (1, 1 << 16, LOW), (2, 1024, LOW), (5, 16, LOW)]
COUNTS = np.array([1, 2047, 5000, 12345, 100003, 3 * 2048 + 1], np.uint64)


@pytest.mark.parametrize("D,d,source", CASES)
def test_histogram_parity(O, D, d, source):
    ctx = R.Context(16)
    ids, p, q, e, m0 = seeded(ctx, O, 41, len(COUNTS), R.E_UNIFORM, 3, 257)
    s0 = np.ones(len(ids), np.uint64)
    hist = ctx.histogram(ids, COUNTS, D, d, source)
    want, m1, s1 = oracle_hist(O, p, q, e, m0, s0, COUNTS, D, d, source)
    np.testing.assert_array_equal(host(hist), want)
    assert int(want.sum()) == sum(int(c) // D for c in COUNTS)
    for i, x in enumerate(ids):
        assert ctx.get_state(int(x)) == (int(m1[i]), int(s1[i]))
    # the next call continues the streams and adds to the same counters
    ctx.histogram(ids, COUNTS, D, d, source, hist=hist)
    want2, _, _ = oracle_hist(O, p, q, e, m1, s1, COUNTS, D, d, source)
    np.testing.assert_array_equal(host(hist), want + want2)


@pytest.mark.parametrize("modexp,divide,T,L", [
    (R.MODEXP_CRT32, R.DIVIDE_INT, 128, 16), (R.MODEXP_CRT32, R.DIVIDE_RECIP, 256, 8),
    (R.MODEXP_CRT32, R.DIVIDE_HYBRID, 128, 4), (R.MODEXP_CRT32, R.DIVIDE_FP64, 512, 2),
    (R.MODEXP_MONT64, R.DIVIDE_RECIP, 128, 8), (R.MODEXP_MONT64, R.DIVIDE_INT, 64, 2)])
def test_histogram_routes_and_tiles(O, modexp, divide, T, L):
    ctx = R.Context(8, modexp=modexp, divide=divide, threads_per_block=T, numbers_per_thread=L)
    ids, p, q, e, m0 = seeded(ctx, O, 43, 4, R.E_UNIFORM, 3, 65537)
    counts = np.array([70001, 3, 4097, 33333], np.uint64)
    s = np.ones(4, np.uint64)
    m = m0
    for D, d, source in [(3, 100, HIGH), (2, 1024, LOW), (1, 999, HIGH)]:
        hist = ctx.histogram(ids, counts, D, d, source)
        want, m, s = oracle_hist(O, p, q, e, m, s, counts, D, d, source)
        np.testing.assert_array_equal(host(hist), want)


def test_histogram_long_streams_in_pieces(O):
    """Streams cut into pieces (skip-sum pre-pass) keep their tuples whole: pieces start on
    tuple boundaries."""
    ctx = R.Context(4, chunk=1 << 16)
    ids, p, q, e, m0 = seeded(ctx, O, 44, 2, R.E_UNIFORM, 3, 65537)
    counts = np.array([3_000_001, 1_234_567], np.uint64)
    m, s = m0, np.ones(2, np.uint64)
    for D, d, source in [(3, 100, HIGH), (5, 16, LOW), (1, 1 << 20, HIGH)]:
        hist = ctx.histogram(ids, counts, D, d, source)
        want, m, s = oracle_hist(O, p, q, e, m, s, counts, D, d, source)
        np.testing.assert_array_equal(host(hist), want)
        for i, x in enumerate(ids):
            assert ctx.get_state(int(x)) == (int(m[i]), int(s[i]))


def test_histogram_argument_errors(O):
    ctx = R.Context(4)
    ids, p, q, e, m0 = seeded(ctx, O, 45, 2, R.E_SMALLEST, 3, 3)
    before = [ctx.get_state(int(x)) for x in ids]
    h = torch.zeros(1 << 20, dtype=torch.int64, device="cuda")
    for D, d, source in [(0, 10, HIGH), (9, 2, HIGH), (2, 1, HIGH), (1, 10, LOW), (1, 16, 7)]:
        with pytest.raises(R.RsaPrngError):
            ctx.histogram(ids[:1], [10], D, d, source, hist=h)
    # d^D = 2^33 bins: refused by the binding's size check before the library's
    with pytest.raises((R.RsaPrngError, ValueError)):
        ctx.histogram(ids[:1], [10], 3, 1 << 11, HIGH, hist=h)
    # the library itself refuses it too (a 2^20-counter buffer is never touched)
    import ctypes
    rc = R._lib.load().rsaprng_histogram(ctx.h, 1, np.array([ids[0]], np.uint32).ctypes.data_as(
        R._lib.pu32), np.array([10], np.uint64).ctypes.data_as(R._lib.pu64), 3, 1 << 11, HIGH,
        ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == R._lib.CODES["ERR_ARG"]
    with pytest.raises(R.RsaPrngError):
        ctx.histogram([ids[0], ids[0]], [10, 10], 1, 16, HIGH, hist=h)
    with pytest.raises(R.RsaPrngError):
        ctx.histogram([12345], [10], 1, 16, HIGH, hist=h)
    torch.cuda.synchronize()
    assert [ctx.get_state(int(x)) for x in ids] == before
    assert int(h.sum()) == 0
    # empty requests are fine and change nothing
    ctx.histogram(ids, [0, 0], 2, 16, HIGH, hist=h)
    assert int(h.sum()) == 0 and [ctx.get_state(int(x)) for x in ids] == before


def test_histogram_bulk_full_size_frequency(O):
    """The bulk workload (1024 streams x 2^20, e uniform in [3, 65537]) through the
    frequency test with 2^20 bins, compared in full with the oracle."""
    cfg = workload.CONFIGS["bulk_1024x2^20"]
    k, n = cfg["instances"], cfg["count"]
    ctx = R.Context(k, chunk=n)
    ids, p, q, e, m0 = seeded(ctx, O, cfg["master"], k, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    counts = np.full(k, n, np.uint64)
    hist = host(ctx.histogram(ids, counts, 1, 1 << 20, HIGH))
    want, m1, s1 = oracle_hist(O, p, q, e, m0, np.ones(k, np.uint64), counts, 1, 1 << 20, HIGH)
    np.testing.assert_array_equal(hist, want)
    for i in (0, 511, 1023):
        assert ctx.get_state(int(ids[i])) == (int(m1[i]), int(s1[i]))
    chi2, total = R.chi2_uniform(hist)
    dof = (1 << 20) - 1
    assert total == k * n
    assert abs(chi2 / dof - 1.0) < 0.01  # seven standard deviations of chi^2 / dof
