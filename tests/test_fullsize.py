"""Full-size parity for the stream-splitting (substream-major and interleaved), batched and
serving workloads: the batched workload on all of its outputs, the others on sampled outputs
(the oracle computes them one by one), and end states."""
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


def oracle_params(O, seeds, cfg):
    par = [O.params_from_seed(int(s), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"]) for s in seeds]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    m0 = np.array([x[3] % (x[0] * x[1]) for x in par], np.uint64)
    return p, q, e, m0


def test_split_full_size_sampled(O):
    """65536 instances x 32 substreams x 2^16 (u64 + f64, 2 TiB in total), generated in
    slices of 1024 instances into reused buffers. Checked: the first output of every
    substream, every output of one substream per slice, and 32 sampled outputs plus the end
    state of every substream of every 251st instance."""
    cfg = workload.CONFIGS["split_65536x32x2^16"]
    K, MV, N = cfg["instances"], cfg["substreams"], cfg["count"]
    SL = 1024
    ctx = R.Context(K + K * MV, chunk=N)
    seeds = workload.instance_seeds(cfg["master"], K)
    first = ctx.create_seeded(seeds, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    p, q, e, m0 = oracle_params(O, seeds, cfg)
    out_c = torch.empty(SL * MV * N, dtype=torch.int64, device="cuda")
    out_r = torch.empty(SL * MV * N, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(9)
    for s0 in range(0, K, SL):
        kids = np.concatenate([ctx.split(first + i, MV) for i in range(s0, s0 + SL)])
        ctx.generate_batch(kids, np.full(len(kids), N, np.uint64), out_r=out_r, out_c=out_c)
        torch.cuda.synchronize()
        # first output of every substream
        idx = torch.arange(0, SL * MV * N, N, device="cuda")
        g_c = out_c[idx].cpu().numpy().view(np.uint64)
        g_r = out_r[idx].cpu().numpy()
        inst = np.repeat(np.arange(s0, s0 + SL), MV)
        gam = np.tile(np.arange(MV), SL)
        s_start = np.array([O.split_s0(1, A, MV, int(g)) for g in range(MV)], np.uint64)[gam]
        m = m0[inst].copy()
        s = s_start.copy()
        want_c, want_r = O.sample_many(p[inst], q[inst], e[inst], np.full(len(inst), A, np.uint64),
                                       m, s, [[1]] * len(inst))
        assert np.array_equal(g_c, want_c) and np.array_equal(bits(g_r), bits(want_r))
        # one whole substream per slice
        j = int(rng.integers(0, SL * MV))
        i, g = s0 + j // MV, j % MV
        c, r, _, _ = O.generate(int(p[i]), int(q[i]), int(e[i]), int(m0[i]),
                                O.split_s0(1, A, MV, g), N, route=O.ROUTE_DIRECT)
        assert np.array_equal(out_c[j * N:(j + 1) * N].cpu().numpy().view(np.uint64), c)
        assert np.array_equal(bits(out_r[j * N:(j + 1) * N].cpu().numpy()), bits(r))
        # every 251st instance: sampled outputs and end states of all its substreams
        for i in range(s0, s0 + SL):
            if i % 251:
                continue
            ks = [np.unique(np.concatenate([rng.integers(1, N + 1, 31), [N]]))
                  for _ in range(MV)]
            m = np.full(MV, m0[i], np.uint64)
            s = s_start[:MV].copy()
            wc, wr = O.sample_many(np.full(MV, p[i]), np.full(MV, q[i]), np.full(MV, e[i]),
                                   np.full(MV, A, np.uint64), m, s, ks)
            base = (i - s0) * MV * N
            gidx = np.concatenate([base + g * N + k - 1 for g, k in enumerate(ks)]).astype(np.int64)
            t = torch.from_numpy(gidx).cuda()
            assert np.array_equal(out_c[t].cpu().numpy().view(np.uint64), wc)
            assert np.array_equal(bits(out_r[t].cpu().numpy()), bits(wr))
            for g in range(MV):
                assert ctx.get_state(int(kids[(i - s0) * MV + g])) == (int(m[g]), int(s[g]))


def test_split_interleaved_full_size_sampled(O):
    """The same 65536 x 32 x 2^16 workload through the vectorised call, in the launch
    configuration the benchmark times (default tiling, 1024 parents per call, each call's
    output k-major: element g N Mv + k Mv + gamma). Checked: the first output of every
    substream, every output of one substream per slice, and 32 sampled outputs plus the end
    state of every substream of every 251st parent."""
    cfg = workload.CONFIGS["split_65536x32x2^16"]
    K, MV, N = cfg["instances"], cfg["substreams"], cfg["count"]
    SL = 1024
    ctx = R.Context(K + K * MV)
    seeds = workload.instance_seeds(cfg["master"], K)
    first = ctx.create_seeded(seeds, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    p, q, e, m0 = oracle_params(O, seeds, cfg)
    out_c = torch.empty(SL * MV * N, dtype=torch.int64, device="cuda")
    out_r = torch.empty(SL * MV * N, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(10)
    s_start = np.array([O.split_s0(1, A, MV, g) for g in range(MV)], np.uint64)
    for s0 in range(0, K, SL):
        kids = np.stack([ctx.split(first + i, MV) for i in range(s0, s0 + SL)])
        ctx.generate_interleaved(kids, N, out_r=out_r, out_c=out_c)
        torch.cuda.synchronize()
        # first output of every substream: elements g N Mv + gamma
        idx = (torch.arange(SL, device="cuda").repeat_interleave(MV) * (N * MV)
               + torch.arange(MV, device="cuda").repeat(SL))
        g_c = out_c[idx].cpu().numpy().view(np.uint64)
        g_r = out_r[idx].cpu().numpy()
        inst = np.repeat(np.arange(s0, s0 + SL), MV)
        gam = np.tile(np.arange(MV), SL)
        want_c, want_r = O.sample_many(p[inst], q[inst], e[inst], np.full(len(inst), A, np.uint64),
                                       m0[inst].copy(), s_start[gam].copy(), [[1]] * len(inst))
        assert np.array_equal(g_c, want_c) and np.array_equal(bits(g_r), bits(want_r))
        # one whole substream per slice: elements g N Mv + k Mv + gamma, k = 0..N-1
        j = int(rng.integers(0, SL * MV))
        i, g = s0 + j // MV, j % MV
        c, r, _, _ = O.generate(int(p[i]), int(q[i]), int(e[i]), int(m0[i]),
                                O.split_s0(1, A, MV, g), N, route=O.ROUTE_DIRECT)
        sub = torch.arange(N, device="cuda") * MV + (j // MV) * N * MV + g
        assert np.array_equal(out_c[sub].cpu().numpy().view(np.uint64), c)
        assert np.array_equal(bits(out_r[sub].cpu().numpy()), bits(r))
        # every 251st parent: sampled outputs and end states of all its substreams
        for i in range(s0, s0 + SL):
            if i % 251:
                continue
            ks = [np.unique(np.concatenate([rng.integers(1, N + 1, 31), [N]]))
                  for _ in range(MV)]
            m = np.full(MV, m0[i], np.uint64)
            s = s_start.copy()
            wc, wr = O.sample_many(np.full(MV, p[i]), np.full(MV, q[i]), np.full(MV, e[i]),
                                   np.full(MV, A, np.uint64), m, s, ks)
            base = (i - s0) * MV * N
            gidx = np.concatenate([base + (k - 1) * MV + g for g, k in enumerate(ks)]).astype(np.int64)
            t = torch.from_numpy(gidx).cuda()
            assert np.array_equal(out_c[t].cpu().numpy().view(np.uint64), wc)
            assert np.array_equal(bits(out_r[t].cpu().numpy()), bits(wr))
            for g in range(MV):
                assert ctx.get_state(int(kids[i - s0][g])) == (int(m[g]), int(s[g]))
    ctx.close()


def test_batched_full_size_graph(O):
    """100000 instances with lognormal lengths (median 2^14, clipped to [100, 1e7], about
    2^32 outputs, 32 GiB), one plan captured in a CUDA graph after autotuning. Checked: all
    outputs against the oracle's direct route, streamed in runs of instances of about 2^27
    outputs, and every instance's end state."""
    cfg = workload.CONFIGS["batched_1e5_lognormal"]
    K = cfg["instances"]
    lens = workload.lognormal_lengths(cfg["master"], K)
    total = int(lens.sum())
    assert 0.8 * 2**32 < total < 1.25 * 2**32
    ctx = R.Context(K)
    seeds = workload.instance_seeds(cfg["master"], K)
    first = ctx.create_seeded(seeds, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    ids = np.arange(first, first + K, dtype=np.uint32)
    tune_ids = ids[:2000]
    ctx.autotune(tune_ids, lens[:2000], reps=1)
    plan = ctx.plan(ids, lens)
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    plan.capture(out_r=out, stream=st)
    plan.replay(stream=st)
    st.synchronize()
    p, q, e, m = oracle_params(O, seeds, cfg)
    s = np.ones(K, np.uint64)
    offs = np.zeros(K + 1, np.int64)
    offs[1:] = np.cumsum(lens.astype(np.int64))
    i0 = 0
    while i0 < K:
        i1 = int(np.searchsorted(offs, offs[i0] + (1 << 27), side="right"))
        i1 = min(K, max(i1 - 1, i0 + 1))
        sl = slice(i0, i1)
        mm, ss = m[sl].copy(), s[sl].copy()
        _, want = O.generate_many(p[sl], q[sl], e[sl], np.full(i1 - i0, A, np.uint64), mm, ss,
                                  lens[sl], route=O.ROUTE_DIRECT, want_c=False)
        got = out[int(offs[i0]):int(offs[i1])].cpu().numpy()
        bad = np.nonzero(bits(got) != bits(want))[0]
        assert len(bad) == 0, f"instances {i0}..{i1}: {len(bad)} outputs differ"
        for j in range(i1 - i0):
            assert ctx.get_state(int(ids[i0 + j])) == (int(mm[j]), int(ss[j])), i0 + j
        i0 = i1
    plan.close()


def test_serving_full_size_sampled(O):
    """1e6 registered instances; 1500 requests (uniform instance, log-uniform count in
    [2^4, 2^24]) submitted at once against a 16 GiB output budget; sampled outputs of every
    request and all outputs of small requests checked."""
    cfg = workload.CONFIGS["serving_1e6"]
    K = cfg["instances"]
    ctx = R.Context(K)
    seeds = workload.instance_seeds(cfg["master"], K)
    first = ctx.create_seeded(seeds, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    srv = R.Server(ctx, out_budget_bytes=16 << 30, nstreams=3)
    n = 1500
    pick = workload.uniform_indices(51, n, K)
    cnt = workload.loguniform_counts(52, n, lo=16, hi=1 << 24)
    tickets = [srv.submit(first + int(i), int(c)) for i, c in zip(pick, cnt)]
    rng = np.random.default_rng(6)
    pos = {}
    used = sorted(set(int(i) for i in pick))
    sub = {i: O.params_from_seed(int(seeds[i]), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
           for i in used}
    for t, i, c in zip(tickets, pick, cnt):
        i, c = int(i), int(c)
        srv.wait(t, timeout_s=300)
        g = srv.result(t).cpu().numpy()
        srv.release(t)
        start = pos.get(i, 0)
        pos[i] = start + c
        pp, qq, ee, ms = sub[i]
        m, s = O.seek(pp, qq, A, ms % (pp * qq), 1, start)
        if c <= 4096:
            _, r, _, _ = O.generate(pp, qq, ee, m, s, c, want_c=False)
            assert np.array_equal(bits(g), bits(r)), (i, c)
        else:
            ks = np.unique(np.concatenate([rng.integers(1, c + 1, 7), [1, c]]))
            _, wr = O.sample_many([pp], [qq], [ee], [A], np.array([m], np.uint64),
                                  np.array([s], np.uint64), [ks])
            assert np.array_equal(bits(g[ks - 1]), bits(wr)), (i, c)
    st = srv.stats()
    assert st["completed"] == n and st["numbers_done"] == int(cnt.sum())
    srv.close()


def test_single_stream_beyond_2p32(O):
    """One stream longer than 2^32 outputs in one call (34 GB of float64): 64-bit positions
    through planning, the skip-sum pre-pass and the kernels. Checked at the start, across
    the 2^32 boundary, at the end, and in the end state; the oracle walks the stream."""
    ctx = R.Context(2)
    seed = int(workload.instance_seeds(71, 1)[0])
    p, q, e, ms = O.params_from_seed(seed)
    m0 = ms % (p * q)
    i = ctx.create(p, q, e, ms)
    N = (1 << 32) + 4099
    r = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.generate_f64(i, N, r)
    torch.cuda.synchronize()
    _, want, _, _ = O.generate(p, q, e, m0, 1, 5000)
    assert (bits(r[:5000].cpu().numpy()) == bits(want)).all()
    k0 = (1 << 32) - 3
    m, s = O.seek_parallel(p, q, A, m0, 1, k0)
    _, want, m, s = O.generate(p, q, e, m, s, 6)
    assert (bits(r[k0:k0 + 6].cpu().numpy()) == bits(want)).all()
    m, s = O.seek_parallel(p, q, A, m, s, N - (k0 + 6) - 1)
    _, want, m, s = O.generate(p, q, e, m, s, 1)
    assert bits(r[N - 1:].cpu().numpy())[0] == bits(want)[0]
    assert ctx.get_state(i) == (m, s)
    del r
    torch.cuda.empty_cache()
