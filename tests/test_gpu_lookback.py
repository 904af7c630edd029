"""The single-launch plain call (decoupled look-back over the tiles' skip sums).

Sec. IV: the message before a tile is m_0 plus all earlier skips (mod n); in
one launch every block gets that sum from the tiles before it. Outputs and
end states must equal the oracle's bit for bit at every size around the tile
and launch boundaries, on every tiling that has a single-launch kernel, and
equal the chunked path's. A device-side wait that runs out must raise the
context's device error flag (the waits are bounded), leave the context usable,
and fault nothing: the test makes tile 0 publish nothing, so that every later
tile's wait runs out.
"""
import ctypes

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1811_11629_gb300 as R  # noqa: E402

A = R.DEFAULT_ROOT


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def _instance(ctx, O, master, rule=R.E_UNIFORM, lo=3, hi=257):
    p, q, e, ms = O.params_from_seed(int(workload.instance_seeds(master, 1)[0]), rule, lo, hi)
    m0 = ms % (p * q)
    return ctx.create_ex(p, q, e, A, m0, 1), (p, q, e, m0)


def _draw(ctx, i, n, both=True):
    c = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda") if both else None
    r = torch.full((n + 1,), -1.0, dtype=torch.float64, device="cuda")
    if both:
        ctx.generate_both(i, n, c, r)
    else:
        ctx.generate_f64(i, n, r)
    torch.cuda.synchronize()
    assert float(r[n]) == -1.0 and (c is None or int(c[n]) == -1)  # nothing past the end
    return (c[:n].cpu().numpy().view(np.uint64) if both else None), r[:n].cpu().numpy()


@pytest.mark.parametrize("cfg", [
    dict(),                                                    # 128 x 16, CRT, reciprocal
    dict(divide=R.DIVIDE_HYBRID), dict(divide=R.DIVIDE_INT), dict(divide=R.DIVIDE_FP64),
    dict(rounding=2),                                          # exact-rational reading
    dict(threads_per_block=64), dict(threads_per_block=512),
    dict(numbers_per_thread=8),
    dict(numbers_per_thread=8, divide=R.DIVIDE_INT, threads_per_block=512),
    dict(modexp=R.MODEXP_MONT64, numbers_per_thread=8),
    dict(modexp=R.MODEXP_MONT64, numbers_per_thread=8, divide=R.DIVIDE_INT),
])
def test_single_launch_sizes_against_oracle(O, cfg):
    """The configured shapes (the latency shape switched off)."""
    ctx = R.Context(4, lookback=R.LOOKBACK_CONFIGURED, **cfg)
    i, (p, q, e, m0) = _instance(ctx, O, 71)
    k = ctx.config()
    S = k["threads_per_block"] * min(k["numbers_per_thread"],
                                     8 if k["modexp"] == R.MODEXP_MONT64 else 16)
    m, s = m0, 1
    launches = ctx.launches
    sizes = [1, S - 1, S, S + 1, 5 * S + 7, 1_000_003]
    for n in sizes:
        c, r = _draw(ctx, i, n)
        want_c, want_r, m, s = O.generate(p, q, e, m, s, n, a=A)
        if cfg.get("rounding") == 2:  # the exact-rational reading of the division
            want_r = O.unit_exact_many(want_c, p * q)
        bad = np.nonzero(c != want_c)[0]
        assert len(bad) == 0, f"n={n}: c differs at {bad[:5]}"
        assert (r.view(np.uint64) == want_r.view(np.uint64)).all(), f"n={n}: r differs"
        assert ctx.get_state(i) == (m, s)
    assert ctx.launches - launches == len(sizes)  # one launch per call
    assert ctx.device_status() == 0


def _latency_shape(n, sms, exact):
    """The library's latency-mode tile (threads, outputs per thread) for a draw of n."""
    T, L = ctypes.c_int32(), ctypes.c_int32()
    assert R._lib.load().rsaprng_latency_shape(n, sms, int(exact), ctypes.byref(T),
                                               ctypes.byref(L)) == 0
    return T.value, L.value


@pytest.mark.parametrize("rounding", [0, 2])
def test_latency_shape_sizes_against_oracle(O, rounding):
    """The latency shapes (tiles of 128-512 threads x 12-16 outputs, at most one per
    SM; CRT, integer division) for draws that fit one wave of 512 x 16 tiles: around
    the chosen tiles' ends and the wave's end, then the configured shape beyond it."""
    ctx = R.Context(4, rounding=rounding)
    i, (p, q, e, m0) = _instance(ctx, O, 74)
    S = 512 * 16
    m, s = m0, 1
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    sizes = [1, S - 1, S, S + 1, 1_000_000, sm * S, sm * S + 1]
    shapes = set()
    for probe in (100_000, 300_000, 600_000, 800_000, 1_000_000, 1_100_000):
        T, L = _latency_shape(probe, sm, rounding == 2)
        shapes.add(L)
        k = -(-probe // (T * L))
        sizes += [k * T * L - 1, k * T * L, k * T * L + 1]
    assert rounding == 2 or shapes >= {12, 13, 14, 16} or sm != 152
    for n in sizes:
        launches = ctx.launches
        c, r = _draw(ctx, i, n)
        assert ctx.launches - launches == 1
        want_c, want_r, m, s = O.generate(p, q, e, m, s, n, a=A)
        if rounding == 2:
            want_r = O.unit_exact_many(want_c, p * q)
        assert (c == want_c).all(), f"n={n}: c differs"
        assert (r.view(np.uint64) == want_r.view(np.uint64)).all(), f"n={n}: r differs"
        assert ctx.get_state(i) == (m, s)
    assert ctx.device_status() == 0


def test_single_launch_limit_and_chunked_path_agree(O):
    """At 4096 tiles the call is one launch; one more output takes the chunked path; with
    the single launch switched off the same draws give the same bits."""
    a = R.Context(4, lookback=R.LOOKBACK_CONFIGURED)
    b = R.Context(4, lookback=R.LOOKBACK_OFF)
    ia, prm = _instance(a, O, 72, R.E_SMALLEST, 3, 3)
    ib, _ = _instance(b, O, 72, R.E_SMALLEST, 3, 3)
    S = 128 * 16
    for n in (4096 * S, 4096 * S + 1, 3_000_000):
        la = a.launches
        _, ra = _draw(a, ia, n, both=False)
        assert (a.launches - la == 1) == (n <= 4096 * S)
        _, rb = _draw(b, ib, n, both=False)
        assert (ra.view(np.uint64) == rb.view(np.uint64)).all()
        assert a.get_state(ia) == b.get_state(ib)
    p, q, e, m0 = prm
    idx = np.array([1, 2, S, S + 1, 1_000_000, 2_999_999, 3_000_000])
    # the last draw's outputs, sampled: output k of that draw is output
    # 2 * 4096 S + 1 + k of the stream
    before = 2 * 4096 * S + 1
    cs, rs = O.sample_many([p], [q], [e], [A], np.array([m0], np.uint64),
                           np.ones(1, np.uint64), [before + idx])
    assert (ra[idx - 1].view(np.uint64) == rs.view(np.uint64)).all()


@pytest.mark.parametrize("spin_limit", [-1, 1000])
def test_wait_that_runs_out_raises_the_device_flag(O, spin_limit):
    ctx = R.Context(4)
    i, (p, q, e, m0) = _instance(ctx, O, 73)
    assert ctx.device_status() == 0
    ctx.configure(spin_limit=spin_limit, test_flags=1)  # tile 0 publishes nothing
    r = torch.empty(1_000_000, dtype=torch.float64, device="cuda")
    ctx.generate_f64(i, 1_000_000, r)  # asynchronous: returns before the waits run out
    assert ctx.device_status() == R._lib.CODES["ERR_DEVICE_FLAG"]
    assert ctx.device_status() == 0  # read and cleared
    # the context stays usable: restore the state and draw again
    ctx.configure()
    ctx.set_state(i, m0, 1)
    c, r2 = _draw(ctx, i, 300_000)
    want_c, want_r, m, s = O.generate(p, q, e, m0, 1, 300_000, a=A)
    assert (c == want_c).all() and (r2.view(np.uint64) == want_r.view(np.uint64)).all()
    assert ctx.get_state(i) == (m, s)
    assert ctx.device_status() == 0
