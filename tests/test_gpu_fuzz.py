"""Randomised parity across the library's entry points: random routes, divisions,
readings of the division, tilings and chunk caps; instances of every mode (default and
small multipliers, constant skips, CRT exponents); the same instances driven through
batched generation, the histogram consumer and the vectorised call in turn, each checked
against the oracle, whose stream states are carried from call to call.
"""
import math
import random

import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1811_11629_gb300 as R  # noqa: E402

Q = (1 << 63) - 25
ROOTS = [R.DEFAULT_ROOT, 3157107955, 3, 7, 11]


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


class Inst:
    """An instance and the oracle's view of its stream."""

    def __init__(self, O, ctx, rng, crt_ok):
        p, q, e, ms = O.params_from_seed(rng.getrandbits(64), R.E_UNIFORM, 3, 4099)
        self.p, self.q, self.e, self.n = p, q, e, p * q
        self.m = rng.randrange(self.n)
        kind = rng.choice(["plain", "constant", "crt"] if crt_ok else ["plain", "constant"])
        self.eq = 0
        if kind == "constant":
            self.a, self.s = 1, rng.randrange(1, Q)
            self.id = ctx.create_ex(p, q, e, 1, self.m, self.s)
        elif kind == "crt":
            self.a, self.s = rng.choice(ROOTS), rng.randrange(1, Q)
            ep = next(x for x in range(rng.randrange(3, 200) | 1, 100000, 2)
                      if math.gcd(x, p - 1) == 1)
            eq = next(x for x in range(rng.randrange(3, 200) | 1, 100000, 2)
                      if math.gcd(x, q - 1) == 1 and x != ep)
            self.e, self.eq = ep, eq
            self.id = ctx.create_crt(p, q, ep, eq, self.a, self.m, self.s)
        else:
            self.a, self.s = rng.choice(ROOTS), rng.randrange(1, Q)
            self.id = ctx.create_ex(p, q, e, self.a, self.m, self.s)

    def take(self, O, count, exact):
        """The next count outputs (c, r) by the oracle; advances the oracle state."""
        c, r, self.m, self.s = O.generate(self.p, self.q, self.e, self.m, self.s, count, a=self.a,
                                          eq=self.eq)
        if exact:
            r = O.unit_exact_many(c, self.n)
        return c, r


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


@pytest.mark.parametrize("seed", range(40))
def test_random_configurations_and_entry_points(O, seed):
    rng = random.Random(1000 + seed)
    modexp = rng.choice([R.MODEXP_CRT32, R.MODEXP_CRT32, R.MODEXP_MONT64])
    T = rng.choice([64, 128, 256, 512])
    L = rng.choice([2, 4, 8] if modexp == R.MODEXP_MONT64 else [2, 4, 8, 16])
    exact = rng.random() < 0.3
    cfg = dict(modexp=modexp, divide=rng.choice([1, 2, 3, 4]), threads_per_block=T,
               numbers_per_thread=L, chunk=rng.choice([0, 1 << 12, 1 << 14, 1 << 16]),
               rounding=R._lib.ROUND_EXACT if exact else R._lib.ROUND_PAPER)
    # the autotuner's knobs (each bit-identical to the default)
    if rng.random() < 0.3 and T // 2 >= 32:
        cfg["streams_per_block"] = 2
    if rng.random() < 0.3:
        cfg["unroll"] = max(1, L // 2)
    cfg["pieces_per_block"] = rng.choice([0, 1, 4])
    cfg = {k: v for k, v in cfg.items() if v}
    ctx = R.Context(32, **cfg)
    insts = [Inst(O, ctx, rng, crt_ok=modexp == R.MODEXP_CRT32) for _ in range(6)]

    # batched generation: requests of random instances (repeats continue the stream)
    picks = [rng.randrange(len(insts)) for _ in range(9)]
    counts = [rng.choice([0, 1, rng.randrange(2, 5000), rng.randrange(5000, 60000)])
              for _ in picks]
    total = sum(counts)
    c_out = torch.empty(max(total, 1), dtype=torch.int64, device="cuda")
    r_out = torch.empty(max(total, 1), dtype=torch.float64, device="cuda")
    ctx.generate_batch([insts[i].id for i in picks], counts, out_r=r_out, out_c=c_out)
    torch.cuda.synchronize()
    gc = c_out.cpu().numpy().view(np.uint64)
    gr = r_out.cpu().numpy()
    off = 0
    for i, n in zip(picks, counts):
        c, r = insts[i].take(O, n, exact)
        np.testing.assert_array_equal(gc[off:off + n], c)
        assert (bits(gr[off:off + n]) == bits(r)).all()
        off += n

    # histogram consumer on distinct instances
    D, d = rng.choice([(1, 4096), (2, 64), (3, 10), (5, 8)])
    low = rng.random() < 0.3 and (d & (d - 1)) == 0
    sel = rng.sample(range(len(insts)), 3)
    hcounts = [rng.randrange(0, 40000) for _ in sel]
    hist = ctx.histogram([insts[i].id for i in sel], hcounts, D, d,
                         R.HIST_LOW if low else R.HIST_HIGH)
    torch.cuda.synchronize()
    want = np.zeros(d ** D, np.uint64)
    for i, n in zip(sel, hcounts):
        c, r = insts[i].take(O, n, exact)
        g = (c % np.uint64(d)).astype(np.int64) if low else \
            np.array([O.digit_of_unit(float(x), d) for x in r], np.int64)
        t = n // D
        if t:
            b = np.zeros(t, np.int64)
            for j in range(D):
                b += g[j:D * t:D] * d ** j
            np.add.at(want, b, 1)
    np.testing.assert_array_equal(hist.cpu().numpy().view(np.uint64), want)

    # the vectorised call on distinct instances
    sel = rng.sample(range(len(insts)), rng.randrange(1, 5))
    N = rng.randrange(1, 30000)
    vr = torch.empty(N * len(sel), dtype=torch.float64, device="cuda")
    ctx.generate_interleaved([insts[i].id for i in sel], N, out_r=vr)
    torch.cuda.synchronize()
    got = vr.cpu().numpy()
    for g, i in enumerate(sel):
        _, r = insts[i].take(O, N, exact)
        assert (bits(got[g::len(sel)]) == bits(r)).all()

    # the direct one-instance call: one launch (latency or configured shape) or the
    # chunked path
    ctx.configure(lookback=rng.choice([R.LOOKBACK_AUTO, R.LOOKBACK_CONFIGURED, R.LOOKBACK_OFF]))
    i = rng.randrange(len(insts))
    N = rng.choice([1, rng.randrange(2, 70000), rng.randrange(70000, 1_500_000)])
    dc = torch.empty(N, dtype=torch.int64, device="cuda")
    dr = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.generate_both(insts[i].id, N, dc, dr)
    torch.cuda.synchronize()
    c, r = insts[i].take(O, N, exact)
    np.testing.assert_array_equal(dc.cpu().numpy().view(np.uint64), c)
    assert (bits(dr.cpu().numpy()) == bits(r)).all()
    assert ctx.device_status() == 0

    # every state where the oracle says it is
    for inst in insts:
        assert ctx.get_state(inst.id) == (inst.m, inst.s)
