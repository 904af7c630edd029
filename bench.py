#!/usr/bin/env python
"""Benchmark of the bulk RSA-exponentiation generator on GB300.

Workload (default): plain bulk, 1024 independent instances (seeded 32-bit
prime pairs, e uniform over valid odd values in [3, 65537]), 2^20 float64
outputs per instance per step, one instance per block: 2^30 numbers and
8 GiB of output per step (larger than L2, so no flush is needed).

A step is one pass of the whole hot path over the batch: skip update, message
prefix, encryption, division and store for every output, plus the state
write-back. `value` is Gnumbers/s with the instance table resident on the
device; `e2e` is the same through the C ABI with host output buffers
(rsaprng_generate_batch_host), device->host copies inside the timed region.

`--impl reference` times the CPU oracle (the paper's CRT + Schrage route, OpenMP
over instances) on a bounded sample of the same workload.

Multi-GPU (torchrun): each rank owns its own 1024 instances (weak scaling, no
data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workload  # noqa: E402

METRIC = "Gnumbers/s float64 on 1 GB300, % int-pipe/HBM roofline; served p50/p99 latency"
UNIT = "Gnumbers/s"
WORKLOAD = "bulk_1024x2^20"
FORMS = ("plain", "batched", "served", "fused", "interleaved", "split_full")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the plain / batched / served forms")
    ap.add_argument("--forms", default=",".join(FORMS),
                    help="comma-separated subset of the forms to run (profiling runs)")
    ap.add_argument("--batched-instances", type=int, default=0,
                    help="instances of the batched form (small profiling runs only)")
    ap.add_argument("--split-count", type=int, default=0,
                    help="outputs per substream of the interleaved form (small profiling "
                         "runs only; default 2^16)")
    ap.add_argument("--parents", type=int, default=1024,
                    help="split parents of the interleaved form (small profiling runs only)")
    ap.add_argument("--tune", action="store_true", help="autotune the tiling before timing")
    ap.add_argument("--tune-cache", default="",
                    help="tuning-cache file: loaded before the run if it exists, saved after")
    ap.add_argument("--instances", type=int, default=0,
                    help="override the instance count (small profiling runs only)")
    ap.add_argument("--count", type=int, default=0,
                    help="override numbers per instance (small profiling runs only)")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--per-thread", type=int, default=0)
    ap.add_argument("--pieces-per-block", type=int, default=4,
                    help="load-balance pieces per resident block of the bulk plan (measured "
                         "best on the bulk workload: 4)")
    ap.add_argument("--unroll", type=int, default=0,
                    help="exponentiation chains per pass (0: all of a thread's numbers)")
    ap.add_argument("--streams-per-block", type=int, default=0,
                    help="streams side by side in a block (0: one)")
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="cap on resident generation blocks per SM (0: occupancy limit)")
    ap.add_argument("--modexp", type=int, default=0)
    ap.add_argument("--divide", type=int, default=0)
    ap.add_argument("--e-rule", default="", choices=["", "smallest", "uniform", "at_least"],
                    help="override the exponent rule (experiments only)")
    ap.add_argument("--e-lo", type=int, default=0)
    ap.add_argument("--e-hi", type=int, default=0)
    return ap.parse_args(argv)


# --------------------------------------------------------------------------- distributed
class Dist:
    def __init__(self, backend_gpu: bool):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            if backend_gpu:
                torch.cuda.set_device(self.local_rank)  # before NCCL binds a device
            dist.init_process_group("nccl" if backend_gpu else "gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def rank_seeds(cfg: dict, rank: int) -> np.ndarray:
    """Per-rank instance seeds: rank r owns instances [r k, (r+1) k) of the master stream."""
    k = cfg["instances"]
    return workload.instance_seeds(cfg["master"], k, first=rank * k)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4)
                          if r[5 + j].lower().startswith("active")})
        # samples under load: the top half of the clock readings taken while busy
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- roofline
def imad_slots_per_number(e: int) -> int:
    """Integer-multiply pipe slots the CRT route needs per output (algorithmic count).

    A slot is one 32-bit low multiply (IMAD) per lane; a high-half multiply
    (IMAD.HI) or a widening 32x32->64 multiply (IMAD.WIDE) issues at half that
    rate and counts 2. One 32-bit Montgomery product = widening a*b (2) + low
    m*pinv (1) + high mq*p (2) = 5. Per output: 2 (bitlen(e) + popcount(e) - 1)
    chain products (squarings, multiplies and the final correction, for p and
    q) and the Garner product (1) = 5 (2k + 1) slots; REDC of m for p and q
    (2 x (1 + 2)); the skip a*s mod Q (two widening products and 25*H: 5);
    Garner's h*q (2). The division r = c / n is the method's one floating-point
    step and is not counted (the default route runs it on the FP64 pipe).
    """
    k = e.bit_length() + bin(e).count("1") - 1
    return 5 * (2 * k + 1) + 6 + 5 + 2


# Library microbenchmarks behind the roofline peaks (rsaprng_microbench kinds).
MICROBENCH = {"imad": 0, "ddiv": 1, "imad_wide": 3, "imad_hi": 4, "mont32": 5, "dfma": 6,
              "cvt_u64_f64": 7, "recip_step": 8}
DIVIDE_RECIP, DIVIDE_INT, DIVIDE_FP64, DIVIDE_HYBRID = 4, 1, 2, 3


def measure_peaks(ctx, torch, device: int) -> dict:
    """Device-wide rates (G per second, all lanes) measured by the library's own
    microbenchmarks in this process, plus the unit counts the nominal figures use."""
    rates = {name: round(ctx.microbench(kind), 2) for name, kind in MICROBENCH.items()}
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(device)
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    return {"rates_G_per_s": rates, "sms": props.multi_processor_count, "sm_max_mhz": sm_max,
            "hbm_gbs": float(peaks.get("hbm_gbs") or 6800.0),
            "hbm_source": "MEASURED_PEAKS.json hbm_gbs (copy)" if peaks.get("hbm_gbs")
            else "fallback 6.8 TB/s",
            "nominal_alu_slots": props.multi_processor_count * 64 * sm_max * 1e6 / 1e9}


def fp64_route_rate(pk: dict, divide: int):
    """Outputs per second (G) the FP64 pipe allows for a division route, or None when
    the route does not use it (the integer route)."""
    r = pk["rates_G_per_s"]
    if divide == DIVIDE_RECIP:
        return r["recip_step"]
    if divide == DIVIDE_HYBRID:
        return r["recip_step"] / 0.75  # three outputs in four
    if divide == DIVIDE_FP64:
        return 1.0 / (1.0 / r["ddiv"] + 1.0 / r["cvt_u64_f64"])
    return None


def bounds(pk: dict, numbers: float, slots: float, seconds: float, divide: int,
           bytes_per_number: int) -> dict:
    """The three bounds of one timed form: the integer-multiply pipe (algorithmic IMAD
    slots per output, as Montgomery-product equivalents of 5 slots, against the measured
    Montgomery-product rate), the FP64 pipe (the division route's measured step rate) and
    HBM (output bytes against the measured copy bandwidth). frac is that of the binding one."""
    rate = numbers / seconds / 1e9
    out = {"alu_frac": round(slots / 5 / seconds / 1e9 / pk["rates_G_per_s"]["mont32"], 4),
           "alu_frac_nominal": round(slots / seconds / 1e9 / pk["nominal_alu_slots"], 4),
           "hbm_frac": round(rate * bytes_per_number / pk["hbm_gbs"], 4)}
    fr = fp64_route_rate(pk, divide)
    out["fp64_frac"] = round(rate / fr, 4) if fr else None
    cand = {"alu": out["alu_frac"], "hbm": out["hbm_frac"]}
    if fr:
        cand["fp64"] = out["fp64_frac"]
    out["bound"] = max(cand, key=cand.get)
    out["frac"] = cand[out["bound"]]
    return out


KERNEL_SOURCES = ["paper_1811_11629_gb300/csrc/kernels.cu",
                  "paper_1811_11629_gb300/csrc/device_math.cuh",
                  "paper_1811_11629_gb300/csrc/kernels.cuh",
                  "paper_1811_11629_gb300/csrc/tile.cuh"]
TRAFFIC_PROFILE = "profiles/dram_traffic_bulk_1024x2p20.md"


def measured_traffic(kernel: dict):
    """DRAM bytes per generation launch from the committed ncu capture, or None when the
    kernel sources or its configuration changed since the capture."""
    import hashlib

    try:
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        text = open(os.path.join(ROOT, TRAFFIC_PROFILE)).read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines()
                  if line.startswith(("traffic_bytes_per_launch:", "kernel_sources_sha256:")))
    if fields.get("kernel_sources_sha256", "").strip() != h.hexdigest():
        return None
    if (kernel.get("modexp"), kernel.get("divide"), kernel.get("threads_per_block"),
            kernel.get("numbers_per_thread")) != (1, 4, 128, 16):
        return None
    return int(fields["traffic_bytes_per_launch"])


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except ValueError:
            pass
    return {}


# --------------------------------------------------------------------------- CPU baseline
def cpu_baseline(cfg: dict, seeds: np.ndarray, target_s: float = 10.0) -> dict:
    """The oracle (paper route: Schrage + CRT, OpenMP over instances) on a bounded sample."""
    import oracle

    oracle.build()
    threads = oracle.max_threads()
    k = len(seeds)
    par = [oracle.params_from_seed(int(s), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
           for s in seeds[:k]]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    a = np.full(k, 2307085864, np.uint64)

    def run(n):
        m = np.array([x[3] % (x[0] * x[1]) for x in par], np.uint64)
        s = np.ones(k, np.uint64)
        t0 = time.perf_counter()
        oracle.generate_many(p, q, e, a, m, s, np.full(k, n, np.uint64),
                             route=oracle.ROUTE_PAPER, want_c=False, want_r=True)
        return time.perf_counter() - t0

    pilot_n = 1024
    dt = run(pilot_n)
    n = int(min(cfg["count"], max(pilot_n, pilot_n * target_s / max(dt, 1e-3))))
    dt = run(n)
    return {"value": k * n / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"all {k} instances x first {n} numbers (of {cfg['count']}) each, "
                      f"route=paper (Schrage + CRT), {dt:.1f} s wall"}


def cpu_oracle_form(name: str, target_s: float = 3.0) -> dict:
    """The oracle (paper route) on a bounded sample of a form's own workload, timed on the
    host cores beside the GPU figure: plain (its one instance, the whole 1e6-number call,
    u64 + f64, one core), batched (its first 2000 instances) and the split workload (4096
    parents x 2^16 numbers; substreams differ from their parent only in the skip state, so
    the parents stand for them)."""
    import oracle

    oracle.build()
    key = {"plain_1x1e6": "plain_1x1e6", "batched_1e5_lognormal": "batched_1e5_lognormal",
           "split_interleaved": "split_65536x32x2^16"}[name]
    cfg = workload.CONFIGS[key]
    k = {"plain_1x1e6": 1, "batched_1e5_lognormal": 2000, "split_interleaved": 4096}[name]
    cap = cfg["count"] if name != "batched_1e5_lognormal" else 1 << 30
    both = name != "batched_1e5_lognormal"
    seeds = workload.instance_seeds(cfg["master"], k)
    par = [oracle.params_from_seed(int(s), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
           for s in seeds]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    a = np.full(k, 2307085864, np.uint64)

    def run(n):
        m = np.array([x[3] % (x[0] * x[1]) for x in par], np.uint64)
        s = np.ones(k, np.uint64)
        t0 = time.perf_counter()
        oracle.generate_many(p, q, e, a, m, s, np.full(k, n, np.uint64),
                             route=oracle.ROUTE_PAPER, want_c=both, want_r=True)
        return time.perf_counter() - t0

    pilot = 8192
    dt = run(pilot)
    n = int(min(cap, max(pilot, pilot * target_s / max(dt, 1e-3))))
    dt = run(n)
    cores = 1 if k == 1 else min(k, oracle.max_threads())
    return {"value": round(k * n / dt / 1e9, 5), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{k} instance(s) of the workload x {n} numbers each"
                      f"{' (u64 + f64)' if both else ''}, route=paper, {dt:.2f} s wall"}


# --------------------------------------------------------------------------- other forms
TUNED_KEYS = ("modexp", "divide", "threads_per_block", "numbers_per_thread", "blocks_per_sm",
              "chunk", "streams_per_block", "unroll", "pieces_per_block")


def _slots(es, counts) -> float:
    return float(sum(imad_slots_per_number(int(e)) * int(c) for e, c in zip(es, counts)))


def form_plain(R, torch, device, pk, rank) -> dict:
    """Plain method: one instance, 1e6 outputs as uint64 c_k and float64 r_k per call."""
    cfg = workload.CONFIGS["plain_1x1e6"]
    ctx = R.Context(4, device=device)
    first = ctx.create_seeded(workload.instance_seeds(cfg["master"], 1, first=rank),
                              cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    n = cfg["count"]
    oc = torch.empty(n, dtype=torch.int64, device="cuda")
    orr = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.generate_both(first, n, oc, orr)
    # five groups of 40 calls, the median group's mean (a call takes about 23 us, so a
    # single short group moves with the launch queue's state)
    reps, groups = 40, []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            ctx.generate_both(first, n, oc, orr)
        b.record()
        torch.cuda.synchronize()
        groups.append(a.elapsed_time(b) / 1e3 / reps)
    dt = sorted(groups)[len(groups) // 2]
    e = ctx.params(first)[2]
    divide = ctx.config()["divide"]
    # A 1e6 draw fits one wave of 512 x 16 tiles, so it runs in a latency shape: at most
    # one tile per SM, 12-16 outputs per thread (512 x 13 on 152 SMs), integer division.
    out = {"value": round(n / dt / 1e9, 3), "unit": UNIT, "ms_per_call": round(dt * 1e3, 4),
           "ms_per_call_of_groups": [round(g * 1e3, 4) for g in groups],
           "e": e, "outputs": "u64+f64", "divide": DIVIDE_INT,
           "hbm_GBps": round(16 * n / dt / 1e9, 1)}
    out.update(bounds(pk, n, _slots([e], [n]), dt, DIVIDE_INT, 16))
    out["path"] = ("one launch, decoupled look-back over the tiles' skip sums, latency shape "
                   "(at most one tile per SM, 12-16 outputs per thread, integer division)")
    T, per = ctypes.c_int32(), ctypes.c_int32()
    if ctx.L.rsaprng_latency_shape(n, pk["sms"], 0, ctypes.byref(T), ctypes.byref(per)) == 0:
        out["tile"] = {"threads": T.value, "per_thread": per.value,
                       "tiles": -(-n // (T.value * per.value))}
    # One wave of at most one block per SM, each a short chain of dependent phases: no pipe
    # is the limit (ncu: issue 38 % active, fetch and barrier stalls); the fractions above
    # say how far.
    out["limited_by"] = "latency (one wave; no pipe saturated)"
    # The same calls through the chunked path (skip-sum pre-pass, scan, generation).
    ctx.configure(lookback=R.LOOKBACK_OFF)
    for _ in range(3):
        ctx.generate_both(first, n, oc, orr)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ctx.generate_both(first, n, oc, orr)
    b.record()
    torch.cuda.synchronize()
    dtc = a.elapsed_time(b) / 1e3 / reps
    out["chunked"] = {"value": round(n / dtc / 1e9, 3), "ms_per_call": round(dtc * 1e3, 4),
                      "path": "pre-pass + scan + generation (three launches)"}
    # One launch in the configured (throughput) shape instead of the latency shape.
    ctx.configure(lookback=R.LOOKBACK_CONFIGURED)
    for _ in range(3):
        ctx.generate_both(first, n, oc, orr)
    a.record()
    for _ in range(reps):
        ctx.generate_both(first, n, oc, orr)
    b.record()
    torch.cuda.synchronize()
    dts = a.elapsed_time(b) / 1e3 / reps
    out["configured_shape"] = {"value": round(n / dts / 1e9, 3), "ms_per_call": round(dts * 1e3, 4),
                               "path": "one launch, 128 x 16 reciprocal-division tiles"}
    ctx.configure()
    assert ctx.device_status() == 0
    # The same draw as a plan captured in a CUDA graph (one graph launch per 1e6 outputs).
    plan = ctx.plan([first], [n])
    st = torch.cuda.Stream()
    plan.capture(out_r=orr, out_c=oc, stream=st)
    for _ in range(3):
        plan.replay(stream=st)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        plan.replay(stream=st)
    b.record(st)
    torch.cuda.synchronize()
    dt = a.elapsed_time(b) / 1e3 / reps
    out["graph"] = {"value": round(n / dt / 1e9, 3), "ms_per_call": round(dt * 1e3, 4),
                    "api": "rsaprng_plan_capture + rsaprng_plan_replay",
                    **bounds(pk, n, _slots([e], [n]), dt, divide, 16)}
    plan.close()
    ctx.close()
    return out


def form_batched(R, torch, device, pk, rank, k=0) -> dict:
    """Batched uneven: 1e5 instances, lognormal lengths (~2^32 outputs, f64), one plan in a
    CUDA graph after autotuning on the whole workload (or a tuning-cache hit). k overrides
    the instance count (the first k of the workload; small profiling runs)."""
    cfg = workload.CONFIGS["batched_1e5_lognormal"]
    k = k or cfg["instances"]
    lens = workload.lognormal_lengths(cfg["master"] + 1000 * rank, k)
    ctx = R.Context(k, device=device)
    first = ctx.create_seeded(workload.instance_seeds(cfg["master"], k, first=rank * k),
                              cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    ids = np.arange(first, first + k, dtype=np.uint32)
    tuned, from_cache = ctx.autotune_cached(ids, lens, reps=1)
    plan = ctx.plan(ids, lens)
    total = int(lens.sum())
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    plan.capture(out_r=out, stream=st)
    for _ in range(2):
        plan.replay(stream=st)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record(st)
    for _ in range(reps):
        plan.replay(stream=st)
    b.record(st)
    st.synchronize()
    dt = a.elapsed_time(b) / 1e3 / reps
    es = [ctx.params(int(i))[2] for i in ids]
    res = {"value": round(total / dt / 1e9, 3), "unit": UNIT, "ms_per_replay": round(dt * 1e3, 3),
           "numbers": total, "launches_per_replay": plan.info()["launches"],
           "chunks": plan.info()["chunks"],
           "tuned": {x: tuned[x] for x in TUNED_KEYS if x in tuned},
           "tuned_from_cache": from_cache,
           "tuning": "rsaprng_autotune_cached on the whole workload (routes, tilings, "
                     "unroll, streams per block, blocks per SM, chunk cap)"}
    res.update(bounds(pk, total, _slots(es, lens), dt, ctx.config()["divide"], 8))
    plan.close()
    del out
    ctx.close()
    torch.cuda.empty_cache()
    return res


def form_fused(R, torch, device, pk, rank, k=0, n=0) -> dict:
    """Fused consumer: the bulk workload (1024 x 2^20, e uniform in [3, 65537]) binned into
    the frequency-test histogram (D = 1, 2^20 bins) and the serial-test histogram (D = 2,
    1024^2 bins) inside the generation kernel; nothing is written per output. k and n
    override the instance count and stream length (small profiling runs)."""
    cfg = workload.CONFIGS["bulk_1024x2^20"]
    k, n = k or cfg["instances"], n or cfg["count"]
    ctx = R.Context(k, device=device, chunk=n)
    first = ctx.create_seeded(workload.instance_seeds(cfg["master"], k, first=rank * k),
                              cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    ids = np.arange(first, first + k, dtype=np.uint32)
    counts = np.full(k, n, np.uint64)
    es = [ctx.params(int(i))[2] for i in ids]
    out = {}
    for name, D, d in (("frequency_2^20", 1, 1 << 20), ("serial_2d_1024^2", 2, 1024)):
        hist = torch.zeros(d ** D, dtype=torch.int64, device="cuda")
        ctx.histogram(ids, counts, D, d, R.HIST_HIGH, hist=hist)  # warm-up
        reps = 3
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hist.zero_()
        a.record()
        for _ in range(reps):
            ctx.histogram(ids, counts, D, d, R.HIST_HIGH, hist=hist)
        b.record()
        torch.cuda.synchronize()
        dt = a.elapsed_time(b) / 1e3 / reps
        chi2, tuples = R.chi2_uniform(hist)
        out[name] = {"value": round(k * n / dt / 1e9, 3), "unit": UNIT,
                     "ms_per_call": round(dt * 1e3, 3),
                     "chi2_per_dof": round(chi2 / (d ** D - 1), 5), "tuples": tuples,
                     **bounds(pk, k * n, _slots(es, [n] * k), dt, ctx.config()["divide"], 0)}
        del hist
    ctx.close()
    return out


def form_interleaved(R, torch, device, pk, rank, parents: int = 1024, count: int = 0) -> dict:
    """The vectorised call of Sec. VI: a slice of the split workload (parents x 32 substreams
    x 2^16, e = 3 or the next valid odd, u64 + f64), every parent's k-major vector in one
    call; the substream-major batch over the same children is timed beside it. count
    replaces the 2^16 outputs per substream in small profiling runs."""
    cfg = workload.CONFIGS["split_65536x32x2^16"]
    mv, n = cfg["substreams"], count or cfg["count"]
    ctx = R.Context(parents * (mv + 1), device=device)
    first = ctx.create_seeded(workload.instance_seeds(cfg["master"], parents, first=rank * parents),
                              cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    kids = [ctx.split(first + i, mv) for i in range(parents)]
    per = mv * n
    oc = torch.empty(parents * per, dtype=torch.int64, device="cuda")
    orr = torch.empty(parents * per, dtype=torch.float64, device="cuda")

    groups = np.stack(kids).astype(np.uint32)
    slots = _slots([ctx.params(first + i)[2] for i in range(parents)], [per] * parents)
    divide = ctx.config()["divide"]

    def vector_calls():
        ctx.generate_interleaved(groups, n, out_r=orr, out_c=oc)

    all_ids = groups.reshape(-1)
    counts = np.full(len(all_ids), n, np.uint64)
    out = {}
    for name, fn in (("interleaved", vector_calls),
                     ("substream_major", lambda: ctx.generate_batch(all_ids, counts, out_r=orr,
                                                                    out_c=oc))):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        dt = a.elapsed_time(b) / 1e3
        out[name] = {"value": round(parents * per / dt / 1e9, 3), "unit": UNIT,
                     "ms": round(dt * 1e3, 2), "hbm_GBps": round(16 * parents * per / dt / 1e9, 1),
                     **bounds(pk, parents * per, slots, dt, divide, 16)}
    out["shape"] = f"{parents} parents x {mv} substreams x {n}, u64 + f64, one call"
    ctx.close()
    del oc, orr
    torch.cuda.empty_cache()
    return out


def form_split_full(R, torch, device, pk, rank, slice_parents: int = 1024) -> dict:
    """The whole split workload: 65536 parents x 32 substreams x 2^16 (2^37 outputs, u64 +
    f64 = 2 TiB, more than HBM holds), generated in slices of slice_parents parents into one
    reused output buffer; throughput over all slices, substream-major and interleaved."""
    cfg = workload.CONFIGS["split_65536x32x2^16"]
    parents, mv, n = cfg["instances"], cfg["substreams"], cfg["count"]
    ctx = R.Context(parents * (mv + 1), device=device)
    first = ctx.create_seeded(workload.instance_seeds(cfg["master"], parents, first=rank * parents),
                              cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    kids = np.stack([ctx.split(first + i, mv) for i in range(parents)]).astype(np.uint32)
    per = slice_parents * mv * n
    oc = torch.empty(per, dtype=torch.int64, device="cuda")
    orr = torch.empty(per, dtype=torch.float64, device="cuda")
    counts = np.full(slice_parents * mv, n, np.uint64)
    slots = _slots([ctx.params(first + i)[2] for i in range(parents)], [mv * n] * parents)
    divide = ctx.config()["divide"]

    def substream_major(s):
        ctx.generate_batch(kids[s:s + slice_parents].reshape(-1), counts, out_r=orr, out_c=oc)

    def interleaved(s):
        ctx.generate_interleaved(kids[s:s + slice_parents], n, out_r=orr, out_c=oc)

    out = {}
    for name, fn in (("substream_major", substream_major), ("interleaved", interleaved)):
        fn(0)  # warm-up slice (continues the first slice's streams; the timed pass covers all)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for s in range(0, parents, slice_parents):
            fn(s)
        b.record()
        torch.cuda.synchronize()
        dt = a.elapsed_time(b) / 1e3
        out[name] = {"value": round(parents * mv * n / dt / 1e9, 3), "unit": UNIT,
                     "s": round(dt, 3), "hbm_GBps": round(16 * parents * mv * n / dt / 1e9, 1),
                     **bounds(pk, parents * mv * n, slots, dt, divide, 16)}
    out["shape"] = (f"{parents} parents x {mv} substreams x {n} = 2^37 outputs, u64 + f64, "
                    f"{parents // slice_parents} slices of {slice_parents} parents into one "
                    f"{16 * per // 2**30} GiB buffer")
    ctx.close()
    del oc, orr
    torch.cuda.empty_cache()
    return out


def form_served(R, torch, device, pk, rank,
                loads=(0.1, 0.25, 0.5, 0.75, 0.9, 1.0, 1.2)) -> dict:
    """Serving: 1e6 registered instances, Poisson arrivals, log-uniform counts in
    [2^4, 2^24], 10^4 requests per point; closed-loop capacity first, then open-loop
    replays at fractions of it (overload included), each point the median of three."""
    cfg = workload.CONFIGS["serving_1e6"]
    k = cfg["instances"]
    ctx = R.Context(k, device=device)
    first = ctx.create_seeded(workload.instance_seeds(cfg["master"], k, first=rank * k),
                              cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    nreq = 10000
    pick = first + workload.uniform_indices(61, nreq, k)
    cnt = workload.loguniform_counts(62, nreq, lo=16, hi=1 << 24)
    # The library's default configuration: the autotuner's sample of the request mix
    # (contiguous outputs, counts capped at 2^20) does not rank the tilings as the server's
    # iterations do (its 256 x 16 choice served 94.7 Gnumbers/s against 104.5 for the
    # default), so the served form runs what a server gets without tuning.
    tuned = ctx.config()
    # four streams: measured 105.1 capacity and p99 0.69 ms at half load, against 103.6 and
    # 0.70 with three, 97.5 with two, 104.9 with six and 100.7 with eight
    srv = R.Server(ctx, out_budget_bytes=16 << 30, nstreams=4)
    mean_cnt = float(cnt.mean())
    # capacity: all requests at once (arrival 0), the server batching freely; the median
    # of three replays (one takes about 0.1 s)
    caps = []
    for _ in range(3):
        srv.replay(pick, cnt, np.zeros(nreq), timeout_s=300)
        st0 = srv.stats()
        caps.append(st0["numbers_done"] / max(st0["wall_s"], 1e-9))
    cap_numbers = sorted(caps)[1]
    cap_rate = cap_numbers / mean_cnt
    points = []
    for f in loads:
        rate = f * cap_rate
        arr = workload.poisson_arrivals(63 + int(f * 100), nreq, rate)
        # three replays of the same trace; the one with the median p99 is reported
        runs = []
        for _ in range(3):
            srv.replay(pick, cnt, arr, timeout_s=300)
            runs.append(srv.stats())
        runs.sort(key=lambda s: s["p99_ms"])
        st = runs[1]
        points.append({"load": f, "offered_req_per_s": round(rate, 1),
                       "throughput": round(st["numbers_done"] / st["wall_s"] / 1e9, 3),
                       "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                       "p99_ms_of_replays": [round(s["p99_ms"], 3) for s in runs],
                       "iterations": st["iterations"],
                       "overlapped_iterations": st["overlapped_iterations"],
                       "submitted": st["submitted"], "admitted": st["admitted"],
                       "completed": st["completed"], "rejected": st["rejected"],
                       "max_inflight_iterations": st["max_inflight_iterations"]})
    es = [ctx.params(int(i))[2] for i in pick[:200]]
    mean_slots = float(np.mean([imad_slots_per_number(int(e)) for e in es]))
    divide = ctx.config()["divide"]
    srv.close()
    ctx.close()
    torch.cuda.empty_cache()
    mid = next((pt for pt in points if pt["load"] == 0.5), points[len(points) // 2])
    return {"value": round(cap_numbers / 1e9, 3), "unit": UNIT,
            "capacity_req_per_s": round(cap_rate, 1), "requests_per_point": nreq,
            "capacity_of_replays": [round(x / 1e9, 3) for x in caps],
            "mean_count": round(mean_cnt, 1), "p50_ms": mid["p50_ms"], "p99_ms": mid["p99_ms"],
            "at_load": mid["load"],
            "config": {x: tuned[x] for x in TUNED_KEYS if x in tuned},
            "points": points, **bounds(pk, cap_numbers, cap_numbers * mean_slots, 1.0, divide, 8)}


# --------------------------------------------------------------------------- our arm
def run_ours(args) -> int:
    import torch

    import paper_1811_11629_gb300 as R

    dist = Dist(backend_gpu=True)
    torch.cuda.set_device(dist.local_rank)
    cfg = dict(workload.CONFIGS[WORKLOAD])
    if args.instances:
        cfg["instances"] = args.instances
    if args.count:
        cfg["count"] = args.count
    if args.e_rule:
        cfg["e_rule"] = {"smallest": workload.E_SMALLEST, "uniform": workload.E_UNIFORM,
                         "at_least": workload.E_AT_LEAST}[args.e_rule]
        cfg["e_lo"] = args.e_lo or 3
        cfg["e_hi"] = args.e_hi or cfg["e_lo"]
    k, n = cfg["instances"], cfg["count"]
    seeds = rank_seeds(cfg, dist.rank)
    knobs = {x: y for x, y in (("threads_per_block", args.threads),
                               ("numbers_per_thread", args.per_thread),
                               ("modexp", args.modexp), ("divide", args.divide),
                               ("blocks_per_sm", args.blocks_per_sm),
                               ("pieces_per_block", args.pieces_per_block),
                               ("unroll", args.unroll),
                               ("streams_per_block", args.streams_per_block)) if y}
    ctx = R.Context(k, device=dist.local_rank, chunk=n, **knobs)
    first = ctx.create_seeded(seeds, cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
    ids = np.arange(first, first + k, dtype=np.uint32)
    counts = np.full(k, n, np.uint64)
    es = [ctx.params(int(i))[2] for i in ids]
    pk = measure_peaks(ctx, torch, dist.local_rank)
    if args.tune_cache and os.path.exists(args.tune_cache):
        R._lib.check(ctx.L.rsaprng_autotune_cache_load(args.tune_cache.encode()), "cache load")
    tuned = None
    if args.tune:
        tuned = ctx.autotune(ids, counts, reps=1)
    plan = ctx.plan(ids, counts)
    out = torch.empty(k * n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.launch(out_r=out, stream=stream)
    torch.cuda.synchronize()
    dist.barrier()

    clocks = ClockSampler(dist.local_rank)
    clocks.start()
    launches0 = ctx.launches
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    gen_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for x, y in gen_ev:  # torch creates the CUDA events at their first record
        x.record(stream)
        y.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for (a, b), g in zip(ev, gen_ev):
        a.record(stream)
        plan.launch(out_r=out, stream=stream, gen_events=g)  # g: the generation kernel alone
        b.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    gpu_launches = ctx.launches - launches0
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    step_ms = [a.elapsed_time(b) for a, b in ev]
    gen_ms = [a.elapsed_time(b) for a, b in gen_ev]
    elapsed_max = dist.max(elapsed)
    numbers_per_step = k * n
    total_numbers = dist.sum(float(numbers_per_step * args.steps))
    value = total_numbers / elapsed_max / 1e9

    # Roofline of the generation kernel, timed alone by the events the plan records around
    # it (a step is also a 4-byte ticket reset, the skip-sum pre-pass over the pieces and
    # the start-state scan): three bounds, each against a rate measured in this process
    # (see measure_peaks).
    kern_s = statistics.mean(gen_ms) / 1e3
    ops = sum(imad_slots_per_number(int(e)) for e in es) * n
    cur = ctx.config()
    b = bounds(pk, numbers_per_step, ops, kern_s, cur["divide"], 8)
    rates = pk["rates_G_per_s"]
    fp64_rate = fp64_route_rate(pk, cur["divide"])
    per_bound = {
        "alu": {"achieved": round(ops / 5 / kern_s / 1e9, 2), "peak": rates["mont32"],
                "unit": "G Montgomery-product equivalents/s", "frac": b["alu_frac"],
                "op": "5 integer-multiply-pipe slots (IMAD = 1, IMAD.HI / IMAD.WIDE = 2), the "
                      "cost of one 32-bit Montgomery product",
                "ops_per_step": ops / 5,
                "peak_source": "measured: rsaprng_microbench 32-bit Montgomery product rate"},
        "fp64": {"achieved": round(numbers_per_step / kern_s / 1e9, 2),
                 "peak": round(fp64_rate, 2) if fp64_rate else None,
                 "unit": "G output steps/s", "frac": b["fp64_frac"],
                 "op": "the division route's output step on the FP64 pipe",
                 "peak_source": "measured: rsaprng_microbench output-step rate of the route"},
        "hbm": {"achieved": round(numbers_per_step * 8 / kern_s / 1e9, 1), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": b["hbm_frac"], "peak_source": pk["hbm_source"]}}
    top = per_bound[b["bound"]]

    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_max * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": k, "numbers_per_instance": n,
                   "e": "uniform over valid odd values in [3, 65537]", "output": "float64",
                   "one_instance_per_block": True, "parallelism": f"instances x{dist.world}",
                   "l2": "outputs 8 GiB per step > L2: no flush"},
        "roofline": {"bound": b["bound"], "achieved": top["achieved"], "peak": top["peak"],
                     "unit": top["unit"], "frac": b["frac"], "traffic": None,
                     "kernel_ms": round(kern_s * 1e3, 3),
                     "step_ms_events": round(statistics.mean(step_ms), 3),
                     "bounds": per_bound,
                     "nominal": {"alu_slots_peak": round(pk["nominal_alu_slots"], 1),
                                 "alu_frac": b["alu_frac_nominal"],
                                 "source": f"{pk['sms']} SMs x 64 IMAD lanes/clk x "
                                           f"{pk['sm_max_mhz']:.0f} MHz (unit counts)"},
                     "rates_measured_G_per_s": rates},
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    if tuned:
        result["config"]["tuned"] = {x: tuned[x] for x in TUNED_KEYS if x in tuned}
    result["config"]["kernel"] = {x: cur[x] for x in TUNED_KEYS if x in cur}
    result["config"]["kernel"].update(plan.shape())
    if (k, n) == (workload.CONFIGS[WORKLOAD]["instances"], workload.CONFIGS[WORKLOAD]["count"]):
        result["roofline"]["traffic"] = measured_traffic(result["config"]["kernel"])
    if (k, n) != (workload.CONFIGS[WORKLOAD]["instances"], workload.CONFIGS[WORKLOAD]["count"]) \
            or args.e_rule:
        result["config"]["workload"] = f"bulk_{k}x{n} e={args.e_rule or 'uniform'} " \
                                       "(experiment, not the benchmark workload)"
    del out
    torch.cuda.empty_cache()

    if not args.no_e2e:
        # End to end: the C-ABI call with a pinned host output buffer; the copies of
        # 8 GiB per step to the host are inside the timed region.
        h_out = torch.empty(k * n, dtype=torch.float64, pin_memory=True)
        ctx.generate_batch_host(ids, counts, h_r=h_out)
        dist.barrier()
        x0 = ctx.transfer_bytes()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.generate_batch_host(ids, counts, h_r=h_out)
        dt = dist.max(time.perf_counter() - t0)
        x1 = ctx.transfer_bytes()
        result["e2e"] = {"value": round(total_numbers / dt / 1e9, 4), "unit": UNIT,
                         "h2d_bytes_per_step": (x1[0] - x0[0]) // args.steps,
                         "d2h_bytes_per_step": (x1[1] - x0[1]) // args.steps,
                         "api": "rsaprng_generate_batch_host (pinned host output)"}
        del h_out
    if not args.no_forms:
        # The plain, batched, served, fused and interleaved forms of the same path on this GPU.
        want = set(args.forms.split(","))
        lr, rk = dist.local_rank, dist.rank
        runs = (("plain_1x1e6", "plain", lambda: form_plain(R, torch, lr, pk, rk)),
                ("batched_1e5_lognormal", "batched",
                 lambda: form_batched(R, torch, lr, pk, rk, args.batched_instances)),
                ("serving_1e6", "served", lambda: form_served(R, torch, lr, pk, rk)),
                ("fused_histogram_bulk", "fused",
                 lambda: form_fused(R, torch, lr, pk, rk, args.instances, args.count)),
                ("split_interleaved", "interleaved",
                 lambda: form_interleaved(R, torch, lr, pk, rk, parents=args.parents,
                                          count=args.split_count)),
                ("split_full_65536x32x2^16", "split_full",
                 lambda: form_split_full(R, torch, lr, pk, rk)))
        result["forms"] = {name: fn() for name, key, fn in runs if key in want}
        if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
            for name in ("plain_1x1e6", "batched_1e5_lognormal", "split_interleaved"):
                if name in result["forms"]:
                    result["forms"][name]["cpu_oracle"] = cpu_oracle_form(name)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(cfg, seeds)
    if args.tune_cache:
        R._lib.check(ctx.L.rsaprng_autotune_cache_save(args.tune_cache.encode()), "cache save")
    if dist.rank == 0:
        print(json.dumps(result), flush=True)
    plan.close()
    ctx.close()
    dist.close()
    return 0


# --------------------------------------------------------------------------- reference arm
def run_reference(args) -> int:
    """The oracle on the host cores, on the same workload, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cfg = workload.CONFIGS[WORKLOAD]
    seeds = rank_seeds(cfg, 0)
    threads = oracle.max_threads()
    k = cfg["instances"]
    par = [oracle.params_from_seed(int(s), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])
           for s in seeds[:k]]
    p = np.array([x[0] for x in par], np.uint64)
    q = np.array([x[1] for x in par], np.uint64)
    e = np.array([x[2] for x in par], np.uint64)
    a = np.full(k, 2307085864, np.uint64)
    m = np.array([x[3] % (x[0] * x[1]) for x in par], np.uint64)
    s = np.ones(k, np.uint64)
    per_step = 1 << 14  # numbers per instance per step (bounded sample)

    def step():
        oracle.generate_many(p, q, e, a, m, s, np.full(k, per_step, np.uint64),
                             route=oracle.ROUTE_PAPER, want_c=False, want_r=True)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = k * per_step * args.steps / dt / 1e9
    sample = (f"all {k} instances x {per_step} consecutive numbers per step "
              f"(of {cfg['count']}), route=paper (Schrage + CRT)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": cfg["instances"],
                   "numbers_per_instance": cfg["count"], "output": "float64"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def main(argv=None) -> int:
    args = parse_args(argv)
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("--steps must be >= 1 and --warmup >= 0")
    unknown = set(args.forms.split(",")) - set(FORMS)
    if unknown:
        raise SystemExit(f"unknown forms: {sorted(unknown)} (known: {', '.join(FORMS)})")
    if args.split_count < 0:
        raise SystemExit("--split-count must be >= 0")
    if args.parents < 1:
        raise SystemExit("--parents must be >= 1")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
