"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit-exact.

Every integer output c_k and every double r_k must equal the oracle's bit for
bit (the tolerance is zero: all integer steps are exact and the one floating
point step is a correctly rounded IEEE division).
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


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def seeded(ctx, O, master, k, rule=R.E_SMALLEST, lo=3, hi=3):
    """k instances from workload seeds; returns ids and the oracle's parameters."""
    seeds = workload.instance_seeds(master, k)
    first = ctx.create_seeded(seeds, rule, lo, hi)
    ids = np.arange(first, first + k, dtype=np.uint32)
    par = []
    for i, s in enumerate(seeds):
        p, q, e, ms = O.params_from_seed(int(s), rule, lo, hi)
        assert ctx.params(int(ids[i])) == (p, q, e, A)
        par.append((p, q, e, ms % (p * q)))
    return ids, par


def check_stream(O, prm, m0, s0, got_c, got_r, a=A):
    p, q, e = prm[:3]
    if got_c is not None:
        got_c = np.asarray(got_c).view(np.uint64)
    n = len(got_c) if got_c is not None else len(got_r)
    c, r, m1, s1 = O.generate(p, q, e, m0, s0, n, a=a)
    if got_c is not None:
        bad = np.nonzero(got_c != c)[0]
        assert len(bad) == 0, f"c mismatch at {bad[:5]} (of {n})"
    if got_r is not None:
        bad = np.nonzero(bits(got_r) != bits(r))[0]
        assert len(bad) == 0, f"r mismatch at {bad[:5]} (of {n})"
    return m1, s1


def test_plain_one_instance_1e6_full(O):
    """Plain method: 1 instance, 1e6 outputs as uint64 c_k and float64 r_k."""
    ctx = R.Context(4)
    ids, par = seeded(ctx, O, master=1, k=1)
    N = 1_000_000
    c = torch.empty(N, dtype=torch.int64, device="cuda")
    r = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.generate_both(int(ids[0]), N, c, r)
    torch.cuda.synchronize()
    m1, s1 = check_stream(O, par[0], par[0][3], 1, c.cpu().numpy(), r.cpu().numpy())
    assert ctx.get_state(int(ids[0])) == (m1, s1)
    # the next call continues the stream
    ctx.generate_both(int(ids[0]), 777, c[:777], r[:777])
    torch.cuda.synchronize()
    check_stream(O, par[0], m1, s1, c[:777].cpu().numpy(), r[:777].cpu().numpy())


ROUTES = [(R.MODEXP_CRT32, R.DIVIDE_INT), (R.MODEXP_CRT32, R.DIVIDE_FP64),
          (R.MODEXP_CRT32, R.DIVIDE_HYBRID), (R.MODEXP_MONT64, R.DIVIDE_INT),
          (R.MODEXP_MONT64, R.DIVIDE_FP64), (R.MODEXP_MONT64, R.DIVIDE_HYBRID),
          (R.MODEXP_CRT32, R.DIVIDE_RECIP), (R.MODEXP_MONT64, R.DIVIDE_RECIP)]
TILES = [(128, 2), (128, 8), (256, 4), (512, 2), (512, 8), (256, 8), (128, 16), (256, 16)]


@pytest.mark.parametrize("modexp,divide", ROUTES)
@pytest.mark.parametrize("threads,L", TILES)
def test_routes_and_tilings_ragged(O, modexp, divide, threads, L):
    """Every route and tiling, ragged counts (0, 1, tile-1, tile, tile+1, ...), two calls."""
    ctx = R.Context(16, modexp=modexp, divide=divide, threads_per_block=threads,
                    numbers_per_thread=L, chunk=1 << 20)
    ids, par = seeded(ctx, O, master=11, k=8, rule=R.E_UNIFORM, lo=3, hi=65537)
    tile = threads * L
    counts = np.array([0, 1, 2, tile - 1, tile, tile + 1, 3 * tile + 5, 20011], np.uint64)
    states = [(pr[3], 1) for pr in par]
    for call in range(2):
        total = int(counts.sum())
        out_c = torch.full((total + 1,), 7, dtype=torch.int64, device="cuda")
        out_r = torch.full((total + 1,), -1.0, dtype=torch.float64, device="cuda")
        ctx.generate_batch(ids, counts, out_r=out_r, out_c=out_c)
        torch.cuda.synchronize()
        gc, gr = out_c.cpu().numpy().view(np.uint64), out_r.cpu().numpy()
        assert gc[total] == 7 and gr[total] == -1.0  # nothing written past the end
        off = 0
        for i in range(len(ids)):
            n = int(counts[i])
            states[i] = check_stream(O, par[i], *states[i], gc[off:off + n], gr[off:off + n])
            assert ctx.get_state(int(ids[i])) == states[i]
            off += n


@pytest.mark.parametrize("kinds", ["r", "rc", "c"])
@pytest.mark.parametrize("threads,L", [(128, 16), (512, 16), (64, 2), (256, 8), (128, 4)])
def test_bulk_tensor_stores(O, threads, L, kinds):
    """Full tiles leave by bulk tensor stores of whole 16-element lines (2-D swizzled views
    of the output arrays; two boxes per tile at 512 x 16). Streams that start at an offset
    of 16k + x0 are staged shifted by x0 (one output kind: two staging buffers), each
    tile's last x0 outputs carried into the next tile's first line; other tiles use
    element stores: a piece's first tile when x0 != 0, ragged ends, full last tiles' tails,
    and everything when the arrays are 8 bytes off 16-byte alignment (second call). Two
    output kinds (one buffer): bulk only at multiples of 16. The u64 output alone takes the
    one-kind path too. Offsets 16k, 16k + 6, 16k + 5,
    16k + 11; pieces of several tiles (one block per SM). Bit-exact with the oracle, and
    the gaps between the ranges keep their fill."""
    ctx = R.Context(8, threads_per_block=threads, numbers_per_thread=L, chunk=1 << 20,
                    blocks_per_sm=1)
    ids, par = seeded(ctx, O, master=19, k=4, rule=R.E_UNIFORM, lo=3, hi=257)
    tile = threads * L
    k = max(3, 400000 // tile)
    counts = np.array([k * tile, k * tile + 17, k * tile, k * tile + 3], np.uint64)
    offs, at = [], 0
    for cnt, x0 in zip(counts, (0, 6, 5, 11)):
        at = (at + 15) // 16 * 16 + 16 + x0
        offs.append(at)
        at += int(cnt)
    total = at + 16
    offsets = np.array(offs, np.uint64)
    states = [(pr[3], 1) for pr in par]
    for call, shift in enumerate((0, 1)):
        cbuf = torch.full((total + shift,), 7, dtype=torch.int64, device="cuda")
        rbuf = torch.full((total + shift,), -1.0, dtype=torch.float64, device="cuda")
        out_c = cbuf[shift:] if "c" in kinds else None
        out_r = rbuf[shift:] if "r" in kinds else None
        ctx.generate_batch(ids, counts, out_r=out_r, out_c=out_c, offsets=offsets)
        torch.cuda.synchronize()
        gr = rbuf.cpu().numpy()[shift:]
        gc = cbuf.cpu().numpy().view(np.uint64)[shift:]
        written = np.zeros(total, bool)
        for i in range(len(ids)):
            o, n = offs[i], int(counts[i])
            written[o:o + n] = True
            states[i] = check_stream(O, par[i], *states[i],
                                     gc[o:o + n] if "c" in kinds else None,
                                     gr[o:o + n] if "r" in kinds else None)
            assert ctx.get_state(int(ids[i])) == states[i]
        assert (gr[~written] == -1.0).all() if "r" in kinds else (gr == -1.0).all()
        assert (gc[~written] == 7).all() if "c" in kinds else (gc == 7).all()


@pytest.mark.parametrize("cfg", [
    dict(streams_per_block=2), dict(streams_per_block=4),
    dict(streams_per_block=2, threads_per_block=256), dict(streams_per_block=8, threads_per_block=256),
    dict(streams_per_block=4, divide=R.DIVIDE_INT), dict(streams_per_block=2, modexp=R.MODEXP_MONT64,
                                                        numbers_per_thread=8),
    dict(unroll=8), dict(unroll=8, divide=R.DIVIDE_HYBRID), dict(unroll=8, divide=R.DIVIDE_INT),
    dict(unroll=4, numbers_per_thread=8), dict(unroll=2),  # the last: no variant, all at once
    dict(unroll=8, streams_per_block=2, chunk=4096),
    dict(pieces_per_block=4), dict(pieces_per_block=3, streams_per_block=2),
])
def test_packed_streams_and_chain_passes(O, cfg):
    """The autotuner's knobs: several streams per block (segments of whole warps, pieces of
    different lengths side by side) and exponentiation chains in passes. Uneven requests,
    several per instance, streams cut into pieces, two calls; bit-exact with the oracle."""
    ctx = R.Context(32, **cfg)
    ids, par = seeded(ctx, O, master=14, k=12, rule=R.E_UNIFORM, lo=3, hi=257)
    req = np.concatenate([ids, ids[:5]]).astype(np.uint32)
    counts = np.array([0, 1, 31, 100, 511, 2047, 2048, 4100, 9000, 33333, 150001, 70, 5,
                       777, 20000, 1, 65536], np.uint64)
    states = {int(i): (pr[3], 1) for i, pr in zip(ids, par)}
    pmap = {int(i): pr for i, pr in zip(ids, par)}
    for call in range(2):
        total = int(counts.sum())
        out_c = torch.full((total + 1,), 7, dtype=torch.int64, device="cuda")
        out_r = torch.full((total + 1,), -1.0, dtype=torch.float64, device="cuda")
        ctx.generate_batch(req, counts, out_r=out_r, out_c=out_c)
        torch.cuda.synchronize()
        gc, gr = out_c.cpu().numpy().view(np.uint64), out_r.cpu().numpy()
        assert gc[total] == 7 and gr[total] == -1.0
        off = 0
        for i in range(len(req)):
            iid, n = int(req[i]), int(counts[i])
            states[iid] = check_stream(O, pmap[iid], *states[iid], gc[off:off + n],
                                       gr[off:off + n])
            off += n
        for iid in states:
            assert ctx.get_state(iid) == states[iid]


def test_chunked_streams_and_fifo_requests(O):
    """Long streams cut into chunks (skip-sum pre-pass) and several requests per instance."""
    ctx = R.Context(8, chunk=4096 * 3, threads_per_block=256, numbers_per_thread=4)
    ids, par = seeded(ctx, O, master=12, k=3, rule=R.E_UNIFORM, lo=3, hi=257)
    a, b, c = (int(x) for x in ids)
    req_ids = np.array([a, b, a, c, a, b], np.uint32)
    counts = np.array([50000, 7, 12289, 100003, 1, 40000], np.uint64)
    # scattered, non-overlapping output offsets
    offsets = np.array([300000, 0, 100, 150000, 299990, 50000], np.uint64)
    out = torch.full((400000,), -1.0, dtype=torch.float64, device="cuda")
    ctx.generate_batch(req_ids, counts, out_r=out, offsets=offsets)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    st = {a: (par[0][3], 1), b: (par[1][3], 1), c: (par[2][3], 1)}
    pmap = {a: par[0], b: par[1], c: par[2]}
    for i in range(len(req_ids)):  # array order = stream order per instance
        iid, n, o = int(req_ids[i]), int(counts[i]), int(offsets[i])
        st[iid] = check_stream(O, pmap[iid], *st[iid], None, g[o:o + n])
    for iid in (a, b, c):
        assert ctx.get_state(iid) == st[iid]


def test_single_instance_chunked_long(O):
    ctx = R.Context(2, chunk=8192)
    ids, par = seeded(ctx, O, master=13, k=1, rule=R.E_AT_LEAST, lo=17, hi=17)
    N = 3_000_017
    r = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.generate_f64(int(ids[0]), N, r)
    torch.cuda.synchronize()
    m1, s1 = check_stream(O, par[0], par[0][3], 1, None, r.cpu().numpy())
    assert ctx.get_state(int(ids[0])) == (m1, s1)


def test_checkpoint_resume(O):
    """Sec. IV state {m, s}: generate N, save, generate M; restore, generate M again."""
    ctx = R.Context(4)
    ids, par = seeded(ctx, O, master=14, k=1, rule=R.E_UNIFORM, lo=3, hi=65537)
    i = int(ids[0])
    x = torch.empty(50000, dtype=torch.int64, device="cuda")
    ctx.generate_u64(i, 12345, x)
    saved = ctx.get_state(i)
    y1 = torch.empty(30000, dtype=torch.int64, device="cuda")
    y2 = torch.empty(30000, dtype=torch.int64, device="cuda")
    ctx.generate_u64(i, 30000, y1)
    ctx.set_state(i, *saved)
    ctx.generate_u64(i, 30000, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    whole = torch.empty(42345, dtype=torch.int64, device="cuda")
    ctx.set_state(i, par[0][3], 1)
    ctx.generate_u64(i, 42345, whole)
    torch.cuda.synchronize()
    assert torch.equal(whole[:12345], x[:12345]) and torch.equal(whole[12345:], y1)
    with pytest.raises(R.RsaPrngError):
        ctx.set_state(i, par[0][0] * par[0][1], 1)  # m >= n
    with pytest.raises(R.RsaPrngError):
        ctx.set_state(i, 0, 0)  # s = 0


def test_split_substreams(O):
    """Sec. VI: child gamma keeps m and starts at s a^(gamma floor((Q-1)/Mv))."""
    ctx = R.Context(64)
    ids, par = seeded(ctx, O, master=15, k=1)
    parent = int(ids[0])
    tmp = torch.empty(1000, dtype=torch.int64, device="cuda")
    ctx.generate_u64(parent, 1000, tmp)  # split from a non-initial state
    m, s = ctx.get_state(parent)
    kids = ctx.split(parent, 32)
    assert ctx.get_state(parent) == (m, s)
    n = 5000
    counts = np.full(32, n, np.uint64)
    oc = torch.empty(32 * n, dtype=torch.int64, device="cuda")
    orr = torch.empty(32 * n, dtype=torch.float64, device="cuda")
    ctx.generate_batch(kids, counts, out_r=orr, out_c=oc)
    torch.cuda.synchronize()
    gc, gr = oc.cpu().numpy().view(np.uint64), orr.cpu().numpy()
    for g in range(32):
        s_g = O.split_s0(s, A, 32, g)
        check_stream(O, par[0], m, s_g, gc[g * n:(g + 1) * n], gr[g * n:(g + 1) * n])
    # child 0 continues the parent's own stream
    pc = torch.empty(n, dtype=torch.int64, device="cuda")
    ctx.generate_u64(parent, n, pc)
    torch.cuda.synchronize()
    assert np.array_equal(pc.cpu().numpy().view(np.uint64), gc[:n].view(np.uint64))


def test_cribs_and_one_guard(O):
    """Sec. IV cribs 0, 1, n-1 and the r = 1.0 guard of Sec. V through the full path."""
    ctx = R.Context(8)
    p, q, e, _ = O.params_from_seed(int(workload.instance_seeds(16, 1)[0]))
    n = p * q
    for target, want_r in ((0, 0.0), (1, None), (n - 1, 1.0 - 2.0**-53)):
        m0 = (target - A) % n  # s_1 = a (s_0 = 1), so m_1 = target
        i = ctx.create_ex(p, q, e, A, m0, 1)
        c = torch.empty(3, dtype=torch.int64, device="cuda")
        r = torch.empty(3, dtype=torch.float64, device="cuda")
        ctx.generate_both(i, 3, c, r)
        torch.cuda.synchronize()
        assert int(c.cpu().numpy().view(np.uint64)[0]) == target
        if want_r is not None:
            assert float(r[0]) == want_r
        check_stream(O, (p, q, e), m0, 1, c.cpu().numpy(), r.cpu().numpy())


@pytest.mark.parametrize("divide", [R.DIVIDE_INT, R.DIVIDE_FP64, R.DIVIDE_RECIP])
def test_unit_step_random_and_edges(O, divide):
    """The output step alone on chosen ciphertexts: random, near n, below 2^53, ties."""
    ctx = R.Context(8)
    ids, par = seeded(ctx, O, master=17, k=4)
    rng = np.random.default_rng(3)
    for i, (p, q, e, _) in zip(ids, par):
        n = p * q
        cs = [rng.integers(0, n, 400000, dtype=np.uint64)]
        cs.append(np.uint64(n) - rng.integers(1, 1 << 14, 20000, dtype=np.uint64))
        cs.append(rng.integers(0, 1 << 54, 20000, dtype=np.uint64))
        cs.append(rng.integers(0, 1 << 32, 20000, dtype=np.uint64))  # high word zero
        # every bit length, random significands (the conversion's normalisation shift)
        cs += [rng.integers(1 << (b - 1), 1 << b, 200, dtype=np.uint64)
               for b in range(1, n.bit_length())]
        edge = [0, 1, 2, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 62) - 1, 1 << 62, n - 1,
                n - 2, n >> 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 1]
        edge += [(1 << b) + d for b in range(1, n.bit_length() - 1) for d in (-1, 0, 1)]
        # values whose conversion to double is an exact tie (ties to even), all bit lengths
        for bl in range(54, n.bit_length() + 1):
            for mant in rng.integers(1 << 52, 1 << 53, 64):
                x = (int(mant) << (bl - 53)) | (1 << (bl - 54))
                if x < n:
                    edge.append(x)
        cs.append(np.array(edge, np.uint64))
        c = np.concatenate(cs)
        dc = torch.from_numpy(c.view(np.int64)).cuda().view(torch.uint64)
        dr = torch.empty(len(c), dtype=torch.float64, device="cuda")
        assert ctx.L.rsaprng_unit_f64(ctx.h, int(i), len(c), dc.data_ptr(), dr.data_ptr(),
                                      divide, torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        want = O.unit_many(c, n)
        got = dr.cpu().numpy()
        bad = np.nonzero(bits(got) != bits(want))[0]
        assert len(bad) == 0, f"n={n}: c={c[bad[:3]]} got={got[bad[:3]]} want={want[bad[:3]]}"
        assert (got < 1.0).all() and (got >= 0.0).all()


@pytest.mark.parametrize("divide", [R.DIVIDE_RECIP, R.DIVIDE_INT, R.DIVIDE_HYBRID,
                                    R.DIVIDE_FP64])
def test_unit_step_near_midpoints(O, divide):
    """The default reading RN(RN(c)/RN(n)) where a route could round the wrong way.

    Sec. V, Eq. CodeFloatingPointStep. Ciphertexts are built so that RN(c)/RN(n)
    lies next to a midpoint between neighbouring doubles (down to 2^-106
    relative), for moduli at the edges of the range (just above 2^62, both
    sides of 2^63, just below 2^64, the largest n) and three seeded ones, with
    c both below 2^53 (exact conversion) and above it (rounded conversion).
    Every route, element by element, against the oracle.
    """
    import division_cases as DC

    ctx = R.Context(16)
    mods = [(p, q) for p, q, _ in DC.EDGE_MODULI]
    for s in workload.instance_seeds(23, 3):
        p, q, _, _ = O.params_from_seed(int(s))
        mods.append((p, q))
    stream = torch.cuda.current_stream().cuda_stream
    for k, (p, q) in enumerate(mods):
        n = p * q
        e = next(x for x in range(3, 999, 2) if math.gcd(x, (p - 1) * (q - 1)) == 1)
        i = ctx.create(p, q, e, 1)
        c = DC.near_midpoint_ciphertexts(n, seed=k)
        assert len(c) >= 100000 and (c < (1 << 53)).any() and (c >= (1 << 53)).any()
        dc = torch.from_numpy(c.view(np.int64)).cuda().view(torch.uint64)
        dr = torch.empty(len(c), dtype=torch.float64, device="cuda")
        assert ctx.L.rsaprng_unit_f64(ctx.h, i, len(c), dc.data_ptr(), dr.data_ptr(), divide,
                                      stream) == 0
        torch.cuda.synchronize()
        want = O.unit_many(c, n)
        got = dr.cpu().numpy()
        bad = np.nonzero(bits(got) != bits(want))[0]
        assert len(bad) == 0, f"n={n}: c={c[bad[:3]]} got={got[bad[:3]]} want={want[bad[:3]]}"


def test_large_exponents(O):
    """Exponents up to 2^32 - 1 exercise the top-bit handling of the square-and-multiply loop."""
    ctx = R.Context(16)
    p, q, _, ms = O.params_from_seed(int(workload.instance_seeds(18, 1)[0]))
    phi = (p - 1) * (q - 1)
    es = [e for e in (3, 5, 7, 65537, 65539, (1 << 31) + 11, (1 << 32) - 1, (1 << 32) - 3,
                      2**31 - 1, 1 << 31 | 1, 0xAAAAAAAB, 0x80000001) if e % 2 and
          math.gcd(e, phi) == 1]
    assert len(es) >= 5
    for modexp in (R.MODEXP_CRT32, R.MODEXP_MONT64):
        ctx.configure(modexp=modexp)
        for e in es:
            i = ctx.create(p, q, e, ms)
            c = torch.empty(3000, dtype=torch.int64, device="cuda")
            r = torch.empty(3000, dtype=torch.float64, device="cuda")
            ctx.generate_both(i, 3000, c, r)
            torch.cuda.synchronize()
            check_stream(O, (p, q, e), ms % (p * q), 1, c.cpu().numpy(), r.cpu().numpy())


def test_all_roots(O):
    """Every allowed skip multiplier (restricted primitive roots and the small roots)."""
    ctx = R.Context(32)
    p, q, e, ms = O.params_from_seed(int(workload.instance_seeds(19, 1)[0]))
    roots = [2307085864, 3157107955, 3200261722, 3211103532, 3338736601, 3423977237,
             3465965455, 3474009732, 3512424704, 3, 6, 7, 10, 11]
    ids = [ctx.create_ex(p, q, e, a, ms % (p * q), 12345) for a in roots]
    n = 10000
    out = torch.empty(len(ids) * n, dtype=torch.int64, device="cuda")
    ctx.generate_batch(np.array(ids, np.uint32), np.full(len(ids), n, np.uint64), out_c=out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    for k, a in enumerate(roots):
        check_stream(O, (p, q, e), ms % (p * q), 12345, g[k * n:(k + 1) * n], None, a=a)
    with pytest.raises(R.RsaPrngError):
        ctx.create_ex(p, q, e, 3163786287, 0, 1)  # listed but not a primitive root


def test_plan_graph_replay(O):
    """A plan captured in a CUDA graph: each replay generates the next outputs."""
    ctx = R.Context(64)
    ids, par = seeded(ctx, O, master=20, k=40, rule=R.E_UNIFORM, lo=3, hi=257)
    counts = workload.lognormal_lengths(20, 40, median=3000.0, sigma=1.0, lo=1, hi=50000)
    total = int(counts.sum())
    plan = ctx.plan(ids, counts)
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    plan.capture(out_r=out, stream=s)
    states = [(pr[3], 1) for pr in par]
    for rep in range(2):
        plan.replay(stream=s)
        s.synchronize()
        g = out.cpu().numpy()
        off = 0
        for i in range(len(ids)):
            n = int(counts[i])
            states[i] = check_stream(O, par[i], *states[i], None, g[off:off + n])
            off += n
    info = plan.info()
    assert info["numbers"] == total and info["launches"] >= 1
    plan.close()


def test_plan_graph_replay_persistent_chunked(O):
    """Replays of a plan whose pieces outnumber the resident blocks (the persistent launch and
    its ticket) and whose streams are cut into many chunks (pre-pass, start-state scan and
    generation launched as programmatic dependents): every replay continues every stream."""
    ctx = R.Context(64, chunk=2048)
    ids, par = seeded(ctx, O, master=22, k=40, rule=R.E_UNIFORM, lo=3, hi=257)
    counts = workload.lognormal_lengths(22, 40, median=150000.0, sigma=0.5, lo=2049, hi=400000)
    total = int(counts.sum())
    plan = ctx.plan(ids, counts)
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    plan.capture(out_r=out, stream=s)
    assert plan.shape()["persistent"] == 1
    states = [(pr[3], 1) for pr in par]
    for rep in range(3):
        plan.replay(stream=s)
        s.synchronize()
        g = out.cpu().numpy()
        off = 0
        for i in range(len(ids)):
            n = int(counts[i])
            states[i] = check_stream(O, par[i], *states[i], None, g[off:off + n])
            off += n
    assert plan.info()["chunks"] > 2000
    plan.close()


def test_plan_launch_timed(O):
    """The timed plan launch (events around the generation kernel alone) continues every
    stream exactly as the plain launch does, with the pre-pass and scan before the first
    event; its events bracket a positive time no longer than the whole launch's; a null
    event is an argument error that launches nothing."""
    ctx = R.Context(64, chunk=4096)
    ids, par = seeded(ctx, O, master=24, k=12, rule=R.E_UNIFORM, lo=3, hi=257)
    counts = np.full(len(ids), 50000, np.uint64)
    total = int(counts.sum())
    plan = ctx.plan(ids, counts)
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    states = [(pr[3], 1) for pr in par]
    for rep in range(3):
        whole = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        gen = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        whole[0].record()
        if rep == 1:
            plan.launch(out_r=out)
        else:
            plan.launch(out_r=out, gen_events=gen)
        whole[1].record()
        torch.cuda.synchronize()
        if rep != 1:
            assert 0 < gen[0].elapsed_time(gen[1]) <= whole[0].elapsed_time(whole[1])
        g = out.cpu().numpy()
        for i in range(len(ids)):
            n = int(counts[i])
            states[i] = check_stream(O, par[i], *states[i], None, g[i * n:(i + 1) * n])
    rc = ctx.L.rsaprng_plan_launch_timed(plan.h, out.data_ptr(), None,
                                         torch.cuda.current_stream().cuda_stream, None, None)
    assert rc == R._lib.CODES["ERR_ARG"]
    assert [ctx.get_state(int(i)) for i in ids] == [s_ for s_ in states]
    assert plan.info()["chunks"] > 100
    plan.close()


def test_autotune_bit_identical_and_state_preserved(O):
    ctx = R.Context(64)
    ids, par = seeded(ctx, O, master=21, k=24, rule=R.E_UNIFORM, lo=3, hi=65537)
    counts = np.full(len(ids), 20000, np.uint64)
    before = [ctx.get_state(int(i)) for i in ids]
    chosen = ctx.autotune(ids, counts, reps=1)
    assert [ctx.get_state(int(i)) for i in ids] == before
    assert chosen["threads_per_block"] in (128, 256, 512)
    out = torch.empty(int(counts.sum()), dtype=torch.float64, device="cuda")
    ctx.generate_batch(ids, counts, out_r=out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    for i in range(len(ids)):
        check_stream(O, par[i], par[i][3], 1, None, g[i * 20000:(i + 1) * 20000])


def test_autotune_cache(O, tmp_path):
    """The tuning cache: a miss tunes, the same workload signature hits and applies the same
    knobs at once, and a saved cache loads into a cleared one; outputs stay bit-exact."""
    L = R._lib.load()
    L.rsaprng_autotune_cache_clear()
    ctx = R.Context(64)
    ids, par = seeded(ctx, O, master=24, k=30, rule=R.E_UNIFORM, lo=3, hi=257)
    counts = workload.lognormal_lengths(24, len(ids), median=4000.0, sigma=1.0, lo=100, hi=60000)
    cfg1, hit1 = ctx.autotune_cached(ids, counts, reps=1)
    assert not hit1 and L.rsaprng_autotune_cache_size() == 1
    ctx2 = R.Context(64)
    ids2, _ = seeded(ctx2, O, master=24, k=30, rule=R.E_UNIFORM, lo=3, hi=257)
    cfg2, hit2 = ctx2.autotune_cached(ids2, counts, reps=1)
    assert hit2
    knobs = ("modexp", "divide", "threads_per_block", "numbers_per_thread", "blocks_per_sm",
             "chunk", "streams_per_block", "unroll", "pieces_per_block")
    assert {k: cfg1[k] for k in knobs} == {k: cfg2[k] for k in knobs}
    path = str(tmp_path / "tune.txt")
    assert L.rsaprng_autotune_cache_save(path.encode()) == 0
    L.rsaprng_autotune_cache_clear()
    assert L.rsaprng_autotune_cache_size() == 0
    assert L.rsaprng_autotune_cache_load(path.encode()) == 0
    _, hit3 = ctx2.autotune_cached(ids2, counts, reps=1)
    assert hit3
    total = int(counts.sum())
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    ctx2.generate_batch(ids2, counts, out_r=out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    off = 0
    for i in range(len(ids2)):
        n = int(counts[i])
        check_stream(O, par[i], par[i][3], 1, None, g[off:off + n])
        off += n
    L.rsaprng_autotune_cache_clear()


@pytest.mark.parametrize("r_mem,c_mem", [("pinned", "pageable"), ("pinned", "pinned"),
                                         ("pageable", "pageable")])
def test_generate_batch_host_equals_device(O, r_mem, c_mem):
    """End-to-end form: outputs land in host memory (pinned buffers written by the kernel
    over the link, pageable ones through device slices); same numbers as the device form."""
    ctx = R.Context(32)
    ids, par = seeded(ctx, O, master=22, k=20, rule=R.E_UNIFORM, lo=3, hi=257)
    counts = np.array([1 << 18] * 10 + [12345] * 10, np.uint64)
    total = int(counts.sum())
    h_r = (torch.empty(total, dtype=torch.float64).pin_memory() if r_mem == "pinned"
           else np.empty(total, np.float64))
    h_c = (torch.empty(total, dtype=torch.int64).pin_memory() if c_mem == "pinned"
           else np.empty(total, np.uint64))
    before = ctx.transfer_bytes()
    ctx.generate_batch_host(ids, counts, h_r=h_r, h_c=h_c)
    after = ctx.transfer_bytes()
    assert after[1] - before[1] == 16 * total  # device->host bytes of both outputs
    g = h_r.numpy() if r_mem == "pinned" else h_r
    gc = h_c.numpy().view(np.uint64) if c_mem == "pinned" else h_c
    off = 0
    for i in range(len(ids)):
        n = int(counts[i])
        check_stream(O, par[i], par[i][3], 1, gc[off:off + n], g[off:off + n])
        off += n


def test_microbenchmarks_run():
    ctx = R.Context(1)
    assert ctx.microbench(0) > 100.0  # G IMAD lane-ops/s
    assert ctx.microbench(1) > 1.0  # G double divisions/s
    assert ctx.microbench(2, 1 << 30) > 500.0  # GB/s


def test_bulk_full_size_all_outputs(O):
    """Plain bulk at full size (1024 instances x 2^20 float64, 8 GiB) in the launch
    configuration the benchmark times (whole streams, four pieces per resident block, bulk
    tensor stores): all 2^30 outputs compared with the oracle's direct route, 128 instances
    at a time, and every end state."""
    cfg = workload.CONFIGS["bulk_1024x2^20"]
    k, n = cfg["instances"], cfg["count"]
    ctx = R.Context(k, chunk=n, pieces_per_block=4)
    seeds = workload.instance_seeds(cfg["master"], k)
    first = ctx.create_seeded(seeds, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    ids = np.arange(first, first + k, dtype=np.uint32)
    plan = ctx.plan(ids, np.full(k, n, np.uint64))
    out = torch.empty(k * n, dtype=torch.float64, device="cuda")
    plan.launch(out_r=out)
    torch.cuda.synchronize()
    par = [O.params_from_seed(int(s), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"]) for s in seeds]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    m = np.array([x[3] % (x[0] * x[1]) for x in par], np.uint64)
    s = np.ones(k, np.uint64)
    B = 128
    for i0 in range(0, k, B):
        sl = slice(i0, i0 + B)
        mm, ss = m[sl].copy(), s[sl].copy()
        _, want = O.generate_many(p[sl], q[sl], e[sl], np.full(B, A, np.uint64), mm, ss,
                                  np.full(B, n, np.uint64), route=O.ROUTE_DIRECT, want_c=False)
        got = out[i0 * n:(i0 + B) * n].cpu().numpy()
        bad = np.nonzero(bits(got) != bits(want))[0]
        assert len(bad) == 0, f"instances {i0}..: {len(bad)} outputs differ, first {bad[:3]}"
        for j in range(B):
            assert ctx.get_state(int(ids[i0 + j])) == (int(mm[j]), int(ss[j])), i0 + j
    plan.close()
