"""GB300 bulk generator for the RSA-exponentiation PRNG of arXiv:1811.11629.

The Python layer is a thin binding of the C ABI in include/rsaprng.h (see
``_lib``); PyTorch supplies device memory and streams. All generation runs in
the CUDA kernels of librsaprng.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (DEFAULT_ROOT, DIVIDE_FP64, DIVIDE_HYBRID, DIVIDE_INT, DIVIDE_RECIP, E_AT_LEAST, E_SMALLEST, E_UNIFORM,
                   HIST_HIGH, HIST_LOW, LOOKBACK_AUTO, LOOKBACK_CONFIGURED, LOOKBACK_OFF,
                   MODEXP_CRT32, MODEXP_MONT64, Q, Config, RsaPrngError, Stats, check)

__all__ = ["Context", "Plan", "Server", "Config", "RsaPrngError", "is_prime", "root_allowed",
           "params_from_seed", "Q", "DEFAULT_ROOT", "MODEXP_CRT32", "MODEXP_MONT64",
           "DIVIDE_INT", "DIVIDE_FP64", "DIVIDE_HYBRID", "DIVIDE_RECIP", "E_SMALLEST", "E_UNIFORM", "E_AT_LEAST",
           "HIST_HIGH", "HIST_LOW", "LOOKBACK_AUTO", "LOOKBACK_CONFIGURED", "LOOKBACK_OFF",
           "chi2_uniform"]


def _u64p(a: np.ndarray):
    return a.ctypes.data_as(_lib.pu64)


def _u32p(a: np.ndarray):
    return a.ctypes.data_as(_lib.pu32)


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("output must be a contiguous CUDA tensor")
    return t.data_ptr()


def chi2_uniform(hist) -> tuple:
    """(chi^2, counted tuples) of a histogram against the uniform expectation
    (rsaprng_chi2_uniform); hist is a host array or a tensor (copied to the host)."""
    if hasattr(hist, "cpu"):
        hist = hist.cpu().numpy()
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    chi2 = ctypes.c_double()
    total = ctypes.c_uint64()
    check(_lib.load().rsaprng_chi2_uniform(_u64p(h), len(h), ctypes.byref(chi2),
                                           ctypes.byref(total)), "chi2_uniform")
    return chi2.value, total.value


def is_prime(x: int) -> bool:
    return bool(_lib.load().rsaprng_is_prime(x))


def validate_params(p: int, q: int, e: int, require_safe: bool = False) -> int:
    """0 or the negative error code instance creation would return."""
    return _lib.load().rsaprng_validate_params(p, q, e, int(require_safe))


def root_allowed(a: int) -> bool:
    return bool(_lib.load().rsaprng_root_allowed(a))


def params_from_seed(seed: int, e_rule: int = E_SMALLEST, e_lo: int = 3, e_hi: int = 3):
    p, q, e, ms = (ctypes.c_uint64() for _ in range(4))
    check(_lib.load().rsaprng_params_from_seed(seed, e_rule, e_lo, e_hi, ctypes.byref(p),
                                               ctypes.byref(q), ctypes.byref(e),
                                               ctypes.byref(ms)), "params_from_seed")
    return p.value, q.value, e.value, ms.value


def make_config(**kw) -> Config:
    c = Config()
    c.struct_size = ctypes.sizeof(Config)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


class Context:
    """A device instance table (rsaprng_ctx)."""

    def __init__(self, max_instances: int, device: int = 0, **config):
        self.L = _lib.load()
        h = ctypes.c_void_p()
        cfg = make_config(**config) if config else None
        check(self.L.rsaprng_ctx_create(ctypes.byref(h), device, max_instances,
                                        ctypes.byref(cfg) if cfg is not None else None),
              "ctx_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.L.rsaprng_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration
    def configure(self, **kw):
        c = make_config(**kw)
        check(self.L.rsaprng_ctx_configure(self.h, ctypes.byref(c)), "configure")

    def config(self) -> dict:
        c = Config()
        check(self.L.rsaprng_ctx_get_config(self.h, ctypes.byref(c)), "get_config")
        return {f: getattr(c, f) for f, _ in Config._fields_ if f not in ("reserved",)}

    @property
    def count(self) -> int:
        return self.L.rsaprng_instance_count(self.h)

    @property
    def launches(self) -> int:
        return self.L.rsaprng_launch_count(self.h)

    def transfer_bytes(self):
        """(host->device, device->host) bytes the library has copied so far."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        check(self.L.rsaprng_transfer_bytes(self.h, ctypes.byref(a), ctypes.byref(b)),
              "transfer_bytes")
        return a.value, b.value

    # -- instances
    def create(self, p: int, q: int, e: int, seed: int) -> int:
        out = ctypes.c_uint32()
        check(self.L.rsaprng_instance_create(self.h, p, q, e, seed, ctypes.byref(out)),
              "instance_create")
        return out.value

    def create_ex(self, p, q, e, a, m0, s0) -> int:
        out = ctypes.c_uint32()
        check(self.L.rsaprng_instance_create_ex(self.h, p, q, e, a, m0, s0, ctypes.byref(out)),
              "instance_create_ex")
        return out.value

    def create_crt(self, p, q, e_p, e_q, a, m0, s0) -> int:
        """Instance with CRT exponents e_p (p residue) and e_q (q residue)."""
        out = ctypes.c_uint32()
        check(self.L.rsaprng_instance_create_crt(self.h, p, q, e_p, e_q, a, m0, s0,
                                                 ctypes.byref(out)), "instance_create_crt")
        return out.value

    def exponents(self, id_: int):
        ep, eq = ctypes.c_uint64(), ctypes.c_uint64()
        check(self.L.rsaprng_get_exponents(self.h, id_, ctypes.byref(ep), ctypes.byref(eq)),
              "get_exponents")
        return ep.value, eq.value

    def create_bulk(self, p, q, e, seed) -> int:
        p, q, e, seed = (np.ascontiguousarray(x, dtype=np.uint64) for x in (p, q, e, seed))
        out = ctypes.c_uint32()
        check(self.L.rsaprng_instances_create_bulk(self.h, len(p), _u64p(p), _u64p(q), _u64p(e),
                                                   _u64p(seed), ctypes.byref(out)), "create_bulk")
        return out.value

    def create_seeded(self, seeds, e_rule=E_SMALLEST, e_lo=3, e_hi=3) -> int:
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        out = ctypes.c_uint32()
        check(self.L.rsaprng_instances_create_seeded(self.h, len(seeds), _u64p(seeds), e_rule,
                                                     e_lo, e_hi, ctypes.byref(out)),
              "create_seeded")
        return out.value

    def split(self, parent: int, mv: int) -> np.ndarray:
        out = np.empty(mv, np.uint32)
        check(self.L.rsaprng_split(self.h, parent, mv, _u32p(out)), "split")
        return out

    def get_state(self, id_: int):
        m, s = ctypes.c_uint64(), ctypes.c_uint64()
        check(self.L.rsaprng_get_state(self.h, id_, ctypes.byref(m), ctypes.byref(s)), "get_state")
        return m.value, s.value

    def set_state(self, id_: int, m: int, s: int):
        check(self.L.rsaprng_set_state(self.h, id_, m, s), "set_state")

    def params(self, id_: int):
        v = [ctypes.c_uint64() for _ in range(4)]
        check(self.L.rsaprng_get_params(self.h, id_, *[ctypes.byref(x) for x in v]), "get_params")
        return tuple(x.value for x in v)

    # -- generation (outputs are caller-owned torch CUDA tensors)
    def generate_u64(self, id_, n, out_c, stream=None):
        check(self.L.rsaprng_generate_u64(self.h, id_, n, _dptr(out_c), _stream_ptr(stream)),
              "generate_u64")

    def generate_f64(self, id_, n, out_r, stream=None):
        check(self.L.rsaprng_generate_f64(self.h, id_, n, _dptr(out_r), _stream_ptr(stream)),
              "generate_f64")

    def generate_both(self, id_, n, out_c, out_r, stream=None):
        check(self.L.rsaprng_generate_both(self.h, id_, n, _dptr(out_c), _dptr(out_r),
                                           _stream_ptr(stream)), "generate_both")

    def device_status(self, stream=None) -> int:
        """Waits for the stream; returns the status code of rsaprng_device_status
        (0, or the device-flag error when a device-side wait gave up) and clears it."""
        return self.L.rsaprng_device_status(self.h, _stream_ptr(stream))

    @staticmethod
    def _req(ids, counts, offsets):
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        counts = np.ascontiguousarray(counts, dtype=np.uint64)
        if offsets is None:
            offsets = np.zeros(len(counts), np.uint64)
            if len(counts) > 1:
                offsets[1:] = np.cumsum(counts[:-1], dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        if not (len(ids) == len(counts) == len(offsets)):
            raise ValueError("ids, counts, offsets differ in length")
        return ids, counts, offsets

    def generate_batch(self, ids, counts, out_r=None, out_c=None, offsets=None, stream=None):
        ids, counts, offsets = self._req(ids, counts, offsets)
        check(self.L.rsaprng_generate_batch(self.h, len(ids), _u32p(ids), _u64p(counts),
                                            _u64p(offsets), _dptr(out_r), _dptr(out_c),
                                            _stream_ptr(stream)), "generate_batch")

    def generate_batch_host(self, ids, counts, h_r=None, h_c=None, offsets=None, stream=None):
        """Outputs into HOST numpy arrays or pinned CPU tensors (end to end)."""
        ids, counts, offsets = self._req(ids, counts, offsets)

        def hp(x):
            if x is None:
                return None
            if isinstance(x, np.ndarray):
                return x.ctypes.data
            return x.data_ptr()

        check(self.L.rsaprng_generate_batch_host(self.h, len(ids), _u32p(ids), _u64p(counts),
                                                 _u64p(offsets), hp(h_r), hp(h_c),
                                                 _stream_ptr(stream)), "generate_batch_host")

    def generate_interleaved(self, ids, n, out_r=None, out_c=None, stream=None):
        """The vectorised call (rsaprng_generate_interleaved). ids: one vector (Mv ids)
        or a 2-D array of ngroups vectors; output k of ids[g][j] at element
        g * n * Mv + k * Mv + j of out_r / out_c (CUDA tensors)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        groups, mv = (1, ids.shape[0]) if ids.ndim == 1 else ids.shape
        ids = ids.reshape(-1)
        for t in (out_r, out_c):
            if t is not None and t.numel() < n * len(ids):
                raise ValueError("output shorter than n * ids.size")
        check(self.L.rsaprng_generate_interleaved(self.h, groups, mv, _u32p(ids), n, _dptr(out_r),
                                                  _dptr(out_c), _stream_ptr(stream)),
              "generate_interleaved")

    def histogram(self, ids, counts, D: int, d: int, source: int = 0, hist=None, stream=None):
        """Frequency (D = 1) / serial (D > 1) test histogram of the next counts[i] outputs
        of ids[i] (rsaprng_histogram). hist: CUDA int64 tensor of d**D counters, added to;
        allocated (zeros) when None. Returns hist."""
        import torch

        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        counts = np.ascontiguousarray(counts, dtype=np.uint64)
        if len(ids) != len(counts):
            raise ValueError("ids and counts differ in length")
        bins = int(d) ** int(D)
        if hist is None:
            hist = torch.zeros(bins, dtype=torch.int64, device=f"cuda:{self.device}")
        elif hist.dtype != torch.int64 or hist.numel() < bins:
            raise ValueError(f"hist must be an int64 tensor of at least d**D = {bins} counters")
        check(self.L.rsaprng_histogram(self.h, len(ids), _u32p(ids), _u64p(counts), D, d, source,
                                       _dptr(hist), _stream_ptr(stream)), "histogram")
        return hist

    def plan(self, ids, counts, offsets=None) -> "Plan":
        return Plan(self, ids, counts, offsets)

    def autotune(self, ids, counts, reps: int = 2) -> dict:
        ids, counts, _ = self._req(ids, counts, None)
        c = Config()
        check(self.L.rsaprng_autotune(self.h, len(ids), _u32p(ids), _u64p(counts), reps,
                                      ctypes.byref(c)), "autotune")
        return {f: getattr(c, f) for f, _ in Config._fields_ if f not in ("reserved",)}

    def autotune_cached(self, ids, counts, reps: int = 2):
        """The tuning-cache lookup, tuning on a miss; returns (config dict, from_cache)."""
        ids, counts, _ = self._req(ids, counts, None)
        c = Config()
        hit = ctypes.c_int32()
        check(self.L.rsaprng_autotune_cached(self.h, len(ids), _u32p(ids), _u64p(counts), reps,
                                             ctypes.byref(c), ctypes.byref(hit)),
              "autotune_cached")
        return {f: getattr(c, f) for f, _ in Config._fields_ if f not in ("reserved",)}, \
            bool(hit.value)

    def microbench(self, kind: int, nbytes: int = 0) -> float:
        r = ctypes.c_double()
        check(self.L.rsaprng_microbench(self.h, kind, nbytes, ctypes.byref(r)), "microbench")
        return r.value


class Plan:
    """A device-resident launch plan (rsaprng_plan), optionally captured as a CUDA graph."""

    def __init__(self, ctx: Context, ids, counts, offsets=None):
        self.ctx = ctx
        self.L = ctx.L
        ids, counts, offsets = Context._req(ids, counts, offsets)
        h = ctypes.c_void_p()
        check(self.L.rsaprng_plan_create(ctx.h, len(ids), _u32p(ids), _u64p(counts),
                                         _u64p(offsets), ctypes.byref(h)), "plan_create")
        self.h = h

    def launch(self, out_r=None, out_c=None, stream=None, gen_events=None):
        """gen_events: a pair of torch.cuda.Event(enable_timing=True) recorded right before
        and after the generation kernel (its time alone, after the pre-pass)."""
        if gen_events is None:
            check(self.L.rsaprng_plan_launch(self.h, _dptr(out_r), _dptr(out_c),
                                             _stream_ptr(stream)), "plan_launch")
            return
        a, b = gen_events
        for ev in (a, b):
            if not ev.cuda_event:  # torch creates the CUDA event at its first record
                ev.record()
        check(self.L.rsaprng_plan_launch_timed(self.h, _dptr(out_r), _dptr(out_c),
                                               _stream_ptr(stream), ctypes.c_void_p(a.cuda_event),
                                               ctypes.c_void_p(b.cuda_event)), "plan_launch_timed")

    def capture(self, out_r=None, out_c=None, stream=None):
        check(self.L.rsaprng_plan_capture(self.h, _dptr(out_r), _dptr(out_c), _stream_ptr(stream)),
              "plan_capture")

    def replay(self, stream=None):
        check(self.L.rsaprng_plan_replay(self.h, _stream_ptr(stream)), "plan_replay")

    def info(self):
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(self.L.rsaprng_plan_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
              "plan_info")
        return {"launches": a.value, "numbers": b.value, "chunks": c.value}

    def shape(self):
        v = [ctypes.c_int32() for _ in range(4)]
        check(self.L.rsaprng_plan_shape(self.h, *[ctypes.byref(x) for x in v]), "plan_shape")
        return dict(zip(("grid", "threads", "blocks_per_sm", "persistent"), (x.value for x in v)))

    def close(self):
        if self.h:
            self.L.rsaprng_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (rsaprng_server)."""

    def __init__(self, ctx: Context, out_budget_bytes: int, nstreams: int = 4):
        self.ctx = ctx
        self.L = ctx.L
        h = ctypes.c_void_p()
        check(self.L.rsaprng_server_create(ctx.h, out_budget_bytes, nstreams, ctypes.byref(h)),
              "server_create")
        self.h = h

    def submit(self, id_: int, count: int) -> int:
        t = ctypes.c_uint64()
        check(self.L.rsaprng_server_submit(self.h, id_, count, ctypes.byref(t)), "server_submit")
        return t.value

    def try_submit(self, id_: int, count: int):
        t = ctypes.c_uint64()
        rc = self.L.rsaprng_server_submit(self.h, id_, count, ctypes.byref(t))
        return rc, t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        check(self.L.rsaprng_server_poll(self.h, ticket, ctypes.byref(d)), "server_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        check(self.L.rsaprng_server_wait(self.h, ticket, int(timeout_s * 1e9)), "server_wait")

    def wait_rc(self, ticket: int, timeout_s: float) -> int:
        return self.L.rsaprng_server_wait(self.h, ticket, int(timeout_s * 1e9))

    def result_ptr(self, ticket: int):
        p = ctypes.c_void_p()
        n = ctypes.c_uint64()
        check(self.L.rsaprng_server_result(self.h, ticket, ctypes.byref(p), ctypes.byref(n)),
              "server_result")
        return p.value, n.value

    def result(self, ticket: int, stream=None):
        """Copies a completed ticket's outputs into a new float64 CUDA tensor."""
        import torch

        _, n = self.result_ptr(ticket)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        st = _stream_ptr(stream)
        check(self.L.rsaprng_server_copy(self.h, ticket, _dptr(out) if n else None, st),
              "server_copy")
        # the copy must finish before the ticket is released and its arena reused
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return out

    def release(self, ticket: int):
        check(self.L.rsaprng_server_release(self.h, ticket), "server_release")

    def cancel(self, ticket: int) -> int:
        return self.L.rsaprng_server_cancel(self.h, ticket)

    def stats(self) -> dict:
        s = Stats()
        check(self.L.rsaprng_server_stats(self.h, ctypes.byref(s)), "server_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def replay(self, ids, counts, arrival_s, timeout_s: float = 600.0):
        """Open-loop replay of a request trace (native load generator); returns latencies."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        counts = np.ascontiguousarray(counts, dtype=np.uint64)
        arr = np.ascontiguousarray(np.round(np.asarray(arrival_s) * 1e9), dtype=np.uint64)
        lat = np.zeros(len(ids), np.float64)
        check(self.L.rsaprng_server_replay(self.h, len(ids), _u32p(ids), _u64p(counts),
                                           _u64p(arr), int(timeout_s * 1e9),
                                           lat.ctypes.data_as(_lib.pdbl)), "server_replay")
        return lat

    def replay_keep(self, ids, counts, arrival_s, timeout_s: float = 600.0) -> np.ndarray:
        """The same replay with every result kept; returns the tickets (read each result
        with result(), then release() it)."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        counts = np.ascontiguousarray(counts, dtype=np.uint64)
        arr = np.ascontiguousarray(np.round(np.asarray(arrival_s) * 1e9), dtype=np.uint64)
        tickets = np.zeros(len(ids), np.uint64)
        check(self.L.rsaprng_server_replay_keep(self.h, len(ids), _u32p(ids), _u64p(counts),
                                                _u64p(arr), int(timeout_s * 1e9),
                                                _u64p(tickets)), "server_replay_keep")
        return tickets

    def close(self):
        if self.h:
            self.L.rsaprng_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
