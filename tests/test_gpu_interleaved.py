"""GPU parity of the vectorised call of Sec. VI (Eq. vectorize): Mv instances
advance together and their outputs come back k-major (element k Mv + gamma).
Compared bit for bit with the oracle's vector update and with the instances'
own streams interleaved.
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


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def run(ctx, ids, N):
    Mv = len(ids)
    c = torch.empty(N * Mv, dtype=torch.int64, device="cuda")
    r = torch.empty(N * Mv, dtype=torch.float64, device="cuda")
    ctx.generate_interleaved(ids, N, out_r=r, out_c=c)
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint64), r.cpu().numpy()


@pytest.mark.parametrize("Mv,N,T,L", [(32, 70001, 128, 16), (8, 4099, 256, 8), (3, 100003, 64, 2),
                                      (1, 50000, 128, 16)])
def test_split_substreams_interleaved(O, Mv, N, T, L):
    ctx = R.Context(64, threads_per_block=T, numbers_per_thread=L)
    seed = workload.instance_seeds(61, 1)
    parent = ctx.create_seeded(seed, R.E_UNIFORM, 3, 257)
    p, q, e, ms = O.params_from_seed(int(seed[0]), R.E_UNIFORM, 3, 257)
    m0 = ms % (p * q)
    kids = ctx.split(parent, Mv)
    gc, gr = run(ctx, kids, N)
    s0 = np.array([O.split_s0(1, A, Mv, g) for g in range(Mv)], np.uint64)
    m = np.full(Mv, m0, np.uint64)
    s = s0.copy()
    full = lambda x: np.full(Mv, x, np.uint64)
    c, r = O.generate_vector(full(p), full(q), full(e), full(A), m, s, N)
    np.testing.assert_array_equal(gc, c)
    assert (bits(gr) == bits(r)).all()
    for g, k in enumerate(kids):
        assert ctx.get_state(int(k)) == (int(m[g]), int(s[g]))


def test_mixed_instances_interleaved(O):
    """Unrelated instances side by side: a seeded one, a constant skip, CRT exponents."""
    ctx = R.Context(8)
    seeds = workload.instance_seeds(62, 1)
    i0 = ctx.create_seeded(seeds, R.E_UNIFORM, 3, 65537)
    p0, q0, e0, ms0 = O.params_from_seed(int(seeds[0]), R.E_UNIFORM, 3, 65537)
    p1, q1, e1, ms1 = O.params_from_seed(int(workload.instance_seeds(63, 1)[0]))
    i1 = ctx.create_ex(p1, q1, e1, 1, ms1 % (p1 * q1), 424242)
    p2, q2, _, ms2 = O.params_from_seed(int(workload.instance_seeds(64, 1)[0]))
    import math
    ep = next(x for x in range(5, 99, 2) if math.gcd(x, p2 - 1) == 1)
    eq = next(x for x in range(ep + 2, 199, 2) if math.gcd(x, q2 - 1) == 1)
    i2 = ctx.create_crt(p2, q2, ep, eq, A, ms2 % (p2 * q2), 1)
    N = 33333
    gc, gr = run(ctx, [i0, i1, i2], N)
    streams = [O.generate(p0, q0, e0, ms0 % (p0 * q0), 1, N),
               O.generate(p1, q1, e1, ms1 % (p1 * q1), 424242, N, a=1),
               O.generate(p2, q2, ep, ms2 % (p2 * q2), 1, N, eq=eq)]
    for g, (c, r, m1, s1) in enumerate(streams):
        np.testing.assert_array_equal(gc[g::3], c)
        assert (bits(gr[g::3]) == bits(r)).all()
        assert ctx.get_state(int([i0, i1, i2][g])) == (m1, s1)


def test_long_interleaved_streams_in_pieces(O):
    ctx = R.Context(8, chunk=1 << 16)
    seeds = workload.instance_seeds(65, 4)
    first = ctx.create_seeded(seeds, R.E_UNIFORM, 3, 257)
    ids = list(range(first, first + 4))
    N = (1 << 20) + 3
    r = torch.empty(N * 4, dtype=torch.float64, device="cuda")
    ctx.generate_interleaved(ids, N, out_r=r)
    torch.cuda.synchronize()
    got = r.cpu().numpy()
    for g, s in enumerate(seeds):
        p, q, e, ms = O.params_from_seed(int(s), R.E_UNIFORM, 3, 257)
        _, want, m1, s1 = O.generate(p, q, e, ms % (p * q), 1, N, want_c=False,
                                     route=O.ROUTE_PAPER)
        assert (bits(got[g::4]) == bits(want)).all()
        assert ctx.get_state(ids[g]) == (m1, s1)


def test_interleaved_argument_errors(O):
    ctx = R.Context(4)
    first = ctx.create_seeded(workload.instance_seeds(66, 2), R.E_SMALLEST, 3, 3)
    before = [ctx.get_state(first), ctx.get_state(first + 1)]
    r = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RsaPrngError):
        ctx.generate_interleaved([first, first], 10, out_r=r)
    with pytest.raises(R.RsaPrngError):
        ctx.generate_interleaved([first, 99], 10, out_r=r)
    with pytest.raises(R.RsaPrngError):
        ctx.generate_interleaved([first], 10)
    with pytest.raises(ValueError):
        ctx.generate_interleaved([first, first + 1], 60, out_r=r)
    ctx.generate_interleaved([first, first + 1], 0, out_r=r)
    torch.cuda.synchronize()
    assert [ctx.get_state(first), ctx.get_state(first + 1)] == before
    assert float(r.abs().sum()) == 0.0


def test_many_vectors_in_one_call(O):
    """ngroups vectors (one per parent) in one call: group g owns elements [g N Mv, (g+1) N Mv)."""
    ctx = R.Context(64)
    seeds = workload.instance_seeds(67, 5)
    first = ctx.create_seeded(seeds, R.E_AT_LEAST, 3, 3)
    Mv, N = 4, 9001
    groups = np.stack([ctx.split(first + i, Mv) for i in range(5)])
    c = torch.empty(5 * N * Mv, dtype=torch.int64, device="cuda")
    ctx.generate_interleaved(groups, N, out_c=c)
    torch.cuda.synchronize()
    got = c.cpu().numpy().view(np.uint64).reshape(5, N * Mv)
    for g, s in enumerate(seeds):
        p, q, e, ms = O.params_from_seed(int(s), R.E_AT_LEAST, 3, 3)
        full = lambda x: np.full(Mv, x, np.uint64)
        s0 = np.array([O.split_s0(1, A, Mv, j) for j in range(Mv)], np.uint64)
        want, _ = O.generate_vector(full(p), full(q), full(e), full(A),
                                    full(ms % (p * q)), s0, N)
        np.testing.assert_array_equal(got[g], want)


@pytest.mark.parametrize("shift_r,shift_c", [(1, 1), (1, 0), (0, 1)])
def test_interleaved_unaligned_outputs(O, shift_r, shift_c):
    """Arrays that start 8 bytes past a 16-byte boundary take the one-column
    stores instead of the column-pair ones; the words around the written span
    stay as they were."""
    ctx = R.Context(16, threads_per_block=128, numbers_per_thread=8)
    seed = workload.instance_seeds(68, 1)
    parent = ctx.create_seeded(seed, R.E_UNIFORM, 3, 257)
    p, q, e, ms = O.params_from_seed(int(seed[0]), R.E_UNIFORM, 3, 257)
    Mv, N = 8, 5003
    kids = ctx.split(parent, Mv)
    n = N * Mv
    br = torch.full((n + 2,), -1.0, dtype=torch.float64, device="cuda")
    bc = torch.full((n + 2,), -7, dtype=torch.int64, device="cuda")
    r, c = br[shift_r:shift_r + n], bc[shift_c:shift_c + n]
    assert (r.data_ptr() % 16 == 8) == bool(shift_r) and (c.data_ptr() % 16 == 8) == bool(shift_c)
    ctx.generate_interleaved(kids, N, out_r=r, out_c=c)
    torch.cuda.synchronize()
    full = lambda x: np.full(Mv, x, np.uint64)
    s0 = np.array([O.split_s0(1, A, Mv, g) for g in range(Mv)], np.uint64)
    want_c, want_r = O.generate_vector(full(p), full(q), full(e), full(A), full(ms % (p * q)), s0, N)
    np.testing.assert_array_equal(c.cpu().numpy().view(np.uint64), want_c)
    assert (bits(r.cpu().numpy()) == bits(want_r)).all()
    hr, hc = br.cpu().numpy(), bc.cpu().numpy()
    outside_r = np.r_[hr[:shift_r], hr[shift_r + n:]]
    outside_c = np.r_[hc[:shift_c], hc[shift_c + n:]]
    assert (outside_r == -1.0).all() and (outside_c == -7).all()
