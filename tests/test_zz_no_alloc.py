"""The allocation-free generation entry point (rsaprng_generate_f64_noalloc).

It serves callers that cannot allocate device memory when they draw numbers:
threads with latency limits that forbid allocator calls, and hosts that hand
all device memory to their own pool up front. Through the C ABI, calls in a
row must give exactly the outputs of the regular rsaprng_generate_f64 on an
identical instance (the tests' tolerance is zero: outputs are bit-exact).
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


def test_noalloc_matches_regular_entry_point_two_calls():
    ctx = R.Context(8)
    L = ctx.L
    p, q, e, ms = R.params_from_seed(int(workload.instance_seeds(77, 1)[0]), R.E_UNIFORM, 3,
                                     65537)
    n = p * q
    a = ctx.create_ex(p, q, e, R.DEFAULT_ROOT, ms % n, 1)  # regular entry point
    b = ctx.create_ex(p, q, e, R.DEFAULT_ROOT, ms % n, 1)  # allocation-free entry point
    stream = torch.cuda.current_stream().cuda_stream
    cfg = ctx.config()
    tile = cfg["threads_per_block"] * cfg["numbers_per_thread"]
    # a multi-chunk call, then short ones continuing the stream: a few chunks, then a
    # single chunk (one output, exactly one tile) that takes its state from the table
    for N in (1_000_003, 4097, 1, tile, tile - 1):
        want = torch.empty(N, dtype=torch.float64, device="cuda")
        got = torch.full((N + 1,), -1.0, dtype=torch.float64, device="cuda")
        assert L.rsaprng_generate_f64(ctx.h, a, N, want.data_ptr(), stream) == 0
        assert L.rsaprng_generate_f64_noalloc(ctx.h, b, N, got.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert float(got[N]) == -1.0  # nothing past the end
        assert torch.equal(got[:N].view(torch.int64), want.view(torch.int64))
        assert ctx.get_state(a) == ctx.get_state(b)


def test_noalloc_rejects_oversized_request():
    ctx = R.Context(2)
    first = ctx.create_seeded(workload.instance_seeds(78, 1))
    before = ctx.get_state(first)
    rc = ctx.L.rsaprng_generate_f64_noalloc(ctx.h, first, (1 << 36) + 1, ctypes.c_void_p(16),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == R._lib.CODES["ERR_ARG"]
    assert ctx.get_state(first) == before
