"""Continuous-batching server: results in the mix equal results alone; admission by
output memory; cancellation and time-outs are raised on the host."""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1811_11629_gb300 as R  # noqa: E402


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


def _instances(ctx, O, master, k, rule=R.E_SMALLEST, lo=3, hi=3):
    seeds = workload.instance_seeds(master, k)
    first = ctx.create_seeded(seeds, rule, lo, hi)
    par = [O.params_from_seed(int(s), rule, lo, hi) for s in seeds]
    return np.arange(first, first + k, dtype=np.uint32), par


def test_server_mix_equals_alone(O):
    """Each request's outputs are its instance's next numbers in submission order,
    whatever else is batched with it (checked against the oracle replaying each
    instance alone)."""
    ctx = R.Context(256, chunk=1 << 16)
    ids, par = _instances(ctx, O, master=30, k=120, rule=R.E_UNIFORM, lo=3, hi=257)
    srv = R.Server(ctx, out_budget_bytes=32 << 20, nstreams=3)
    nreq = 500
    pick = workload.uniform_indices(31, nreq, len(ids))
    cnt = workload.loguniform_counts(32, nreq, lo=16, hi=1 << 18)
    tickets = [srv.submit(int(ids[i]), int(c)) for i, c in zip(pick, cnt)]
    got = []
    for t in tickets:
        srv.wait(t, timeout_s=120)
        ptr, n = srv.result_ptr(t)
        assert ptr % 128 == 0  # results start on whole 16-element lines of the arena
        got.append(srv.result(t).cpu().numpy())
        srv.release(t)
    # oracle: each instance alone, requests concatenated in submission order
    per_inst = {}
    for i, c in zip(pick, cnt):
        per_inst[int(i)] = per_inst.get(int(i), 0) + int(c)
    keys = sorted(per_inst)
    p = np.array([par[i][0] for i in keys], np.uint64)
    q = np.array([par[i][1] for i in keys], np.uint64)
    e = np.array([par[i][2] for i in keys], np.uint64)
    a = np.full(len(keys), R.DEFAULT_ROOT, np.uint64)
    m = np.array([par[i][3] % (par[i][0] * par[i][1]) for i in keys], np.uint64)
    s = np.ones(len(keys), np.uint64)
    counts = np.array([per_inst[i] for i in keys], np.uint64)
    _, ref = O.generate_many(p, q, e, a, m, s, counts, route=O.ROUTE_DIRECT, want_c=False)
    start = {}
    off = 0
    for i, n in zip(keys, counts):
        start[i] = off
        off += int(n)
    cursor = dict(start)
    for (i, c), g in zip(zip(pick, cnt), got):
        i, c = int(i), int(c)
        want = ref[cursor[i]:cursor[i] + c]
        cursor[i] += c
        assert np.array_equal(g.view(np.uint64), want.view(np.uint64)), (i, c)
    st = srv.stats()
    assert st["completed"] == nreq and st["submitted"] == nreq
    assert st["numbers_done"] == int(cnt.sum())
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    # the device state ends where the oracle's does
    for j, i in enumerate(keys):
        assert ctx.get_state(int(ids[i])) == (int(m[j]), int(s[j]))


def test_server_admission_budget_cancel_timeout():
    """Admission by output memory; over-budget requests are rejected; a request that
    cannot be admitted times out on the host and can be cancelled."""
    ctx = R.Context(16)
    seeds = workload.instance_seeds(33, 4)
    first = ctx.create_seeded(seeds)
    srv = R.Server(ctx, out_budget_bytes=8 * 10000, nstreams=2)
    rc, _ = srv.try_submit(first, 10001)
    assert rc == R._lib.CODES["ERR_BUDGET"]
    t1 = srv.submit(first, 10000)  # fills the arena
    t2 = srv.submit(first + 1, 5000)  # must wait for t1's release
    srv.wait(t1, timeout_s=60)
    assert srv.wait_rc(t2, 0.2) == R._lib.CODES["ERR_TIMEOUT"]
    assert not srv.poll(t2)
    assert srv.cancel(t2) == 0
    with pytest.raises(R.RsaPrngError):
        srv.poll(t2)
    srv.release(t2)
    srv.release(t1)
    t3 = srv.submit(first + 1, 5000)
    srv.wait(t3, timeout_s=60)
    assert srv.poll(t3)
    with pytest.raises(R.RsaPrngError):
        srv.submit(10_000, 5)  # unknown instance
    st = srv.stats()
    assert st["rejected"] == 1 and st["cancelled"] == 1 and st["completed"] == 2
    srv.release(t3)
    srv.close()


def test_server_replay_open_loop(O):
    """Native open-loop replay: Poisson arrivals, log-uniform sizes, p50/p99 reported."""
    ctx = R.Context(2000)
    ids, _ = _instances(ctx, O, master=34, k=1000)
    srv = R.Server(ctx, out_budget_bytes=256 << 20, nstreams=2)
    n = 2000
    pick = ids[workload.uniform_indices(35, n, len(ids))]
    cnt = workload.loguniform_counts(36, n, lo=16, hi=1 << 20)
    arr = workload.poisson_arrivals(37, n, rate_per_s=20000.0)
    lat = srv.replay(pick, cnt, arr, timeout_s=120)
    st = srv.stats()
    assert st["completed"] == n and st["numbers_done"] == int(cnt.sum())
    assert (lat > 0).all() and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_server_serves_every_mode(O):
    """Constant-skip and CRT-exponent instances through the server, mixed with ordinary ones,
    under the exact-rational reading: every request equals its instance's next numbers."""
    import math

    ctx = R.Context(16, rounding=R._lib.ROUND_EXACT)
    p0, q0, e0, ms0 = O.params_from_seed(int(workload.instance_seeds(33, 1)[0]))
    i0 = ctx.create_ex(p0, q0, e0, 1, ms0 % (p0 * q0), 31337)  # constant skip
    p1, q1, _, ms1 = O.params_from_seed(int(workload.instance_seeds(34, 1)[0]))
    ep = next(x for x in range(5, 99, 2) if math.gcd(x, p1 - 1) == 1)
    eq = next(x for x in range(ep + 2, 199, 2) if math.gcd(x, q1 - 1) == 1)
    i1 = ctx.create_crt(p1, q1, ep, eq, R.DEFAULT_ROOT, ms1 % (p1 * q1), 1)
    p2, q2, e2, ms2 = O.params_from_seed(int(workload.instance_seeds(35, 1)[0]))
    i2 = ctx.create(p2, q2, e2, ms2)
    srv = R.Server(ctx, out_budget_bytes=16 << 20, nstreams=2)
    reqs = [(i0, 70001), (i1, 5000), (i2, 123457), (i0, 3), (i1, 99999), (i2, 1)]
    tickets = [srv.submit(i, n) for i, n in reqs]
    got = {}
    for (i, n), t in zip(reqs, tickets):
        srv.wait(t, timeout_s=120)
        got.setdefault(i, []).append(srv.result(t).cpu().numpy())
        srv.release(t)
    srv.close()
    spec = {i0: (p0, q0, e0, ms0 % (p0 * q0), 31337, 1, 0),
            i1: (p1, q1, ep, ms1 % (p1 * q1), 1, R.DEFAULT_ROOT, eq),
            i2: (p2, q2, e2, ms2 % (p2 * q2), 1, R.DEFAULT_ROOT, 0)}
    for i, (p, q, e, m0, s0, a, eqq) in spec.items():
        seq = np.concatenate(got[i])
        c, _, _, _ = O.generate(p, q, e, m0, s0, len(seq), a=a, eq=eqq)
        want = O.unit_exact_many(c, p * q)
        assert (seq.view(np.uint64) == want.view(np.uint64)).all()


def test_continuous_batching_poisson_arrivals(O):
    """Continuous batching, not a queue: requests arrive (Poisson, paced by the native
    replay) while earlier ones run; iterations overlap on the device (their event
    intervals on different streams overlap); and every request's outputs equal its
    instance's stream at the request's position, replayed alone by the oracle."""
    ctx = R.Context(128)
    ids, par = _instances(ctx, O, master=40, k=64, rule=R.E_UNIFORM, lo=3, hi=257)
    nreq = 1500
    pick = ids[workload.uniform_indices(41, nreq, len(ids))]
    cnt = workload.loguniform_counts(42, nreq, lo=1 << 10, hi=1 << 19)
    arrivals = workload.poisson_arrivals(43, nreq, rate_per_s=200_000.0)
    total = int(cnt.sum())
    srv = R.Server(ctx, out_budget_bytes=8 * total + (1 << 20), nstreams=3)
    tickets = srv.replay_keep(pick, cnt, arrivals, timeout_s=300)
    st = srv.stats()
    assert st["completed"] == nreq
    assert st["max_inflight_iterations"] >= 2
    assert st["overlapped_iterations"] >= 1
    assert st["iterations"] > 1
    got = [srv.result(int(t)).cpu().numpy() for t in tickets]
    for t in tickets:
        srv.release(int(t))
    srv.close()
    # the oracle: each instance alone, its requests concatenated in arrival order
    first = int(ids[0])
    per = {}
    for i, c in zip(pick, cnt):
        per.setdefault(int(i), []).append(int(c))
    keys = sorted(per)
    p = np.array([par[i - first][0] for i in keys], np.uint64)
    q = np.array([par[i - first][1] for i in keys], np.uint64)
    e = np.array([par[i - first][2] for i in keys], np.uint64)
    a = np.full(len(keys), R.DEFAULT_ROOT, np.uint64)
    m = np.array([par[i - first][3] % (par[i - first][0] * par[i - first][1]) for i in keys],
                 np.uint64)
    s = np.ones(len(keys), np.uint64)
    counts = np.array([sum(per[i]) for i in keys], np.uint64)
    _, ref = O.generate_many(p, q, e, a, m, s, counts, route=O.ROUTE_DIRECT, want_c=False)
    start = dict(zip(keys, np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)))
    pos = {i: 0 for i in keys}
    for j, (i, c) in enumerate(zip(pick, cnt)):
        i, c = int(i), int(c)
        o = int(start[i]) + pos[i]
        assert (got[j].view(np.uint64) == ref[o:o + c].view(np.uint64)).all(), f"request {j}"
        pos[i] += c
