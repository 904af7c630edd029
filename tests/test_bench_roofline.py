"""The roofline's algorithmic count (bench.py): integer-multiply slots per output of the CRT
route, checked against counts made by hand from the exponent's square-and-multiply chain,
and the bulk workload's average quoted in the design notes."""
import numpy as np

import bench
import oracle
import workload


def chain_products(e):
    """Montgomery products of left-to-right square-and-multiply for e, per residue."""
    bits = bin(e)[3:]  # after the leading one
    return sum(2 if b == "1" else 1 for b in bits)


def test_slots_by_hand():
    # per output: 5 slots per Montgomery product over 2 (chain + correction) + 1 (Garner)
    # products, 2 x 3 for the reductions of m, 5 for the skip, 2 for Garner's h q
    for e in (3, 5, 7, 17, 257, 65537, 65535, 40961):
        k = chain_products(e) + 1  # the correction product
        assert k == e.bit_length() + bin(e).count("1") - 1
        want = 5 * (2 * k + 1) + 6 + 5 + 2
        assert bench.imad_slots_per_number(e) == want, e
    assert bench.imad_slots_per_number(3) == 48
    assert bench.imad_slots_per_number(65537) == 198


def test_bulk_average():
    cfg = workload.CONFIGS["bulk_1024x2^20"]
    seeds = workload.instance_seeds(cfg["master"], cfg["instances"])
    es = [oracle.params_from_seed(int(s), cfg["e_rule"], cfg["e_lo"], cfg["e_hi"])[2]
          for s in seeds]
    mean = float(np.mean([bench.imad_slots_per_number(int(e)) for e in es]))
    assert abs(mean - 243.5) < 0.5


def _fake_peaks():
    return {"rates_G_per_s": {"mont32": 3500.0, "recip_step": 160.0, "ddiv": 70.0,
                              "cvt_u64_f64": 300.0},
            "hbm_gbs": 6800.0, "nominal_alu_slots": 20000.0}


def test_bounds_pick_the_binding_unit():
    pk = _fake_peaks()
    # bulk-like: 2^30 outputs, 243.5 slots each, 19.7 ms -> the multiply pipe binds
    b = bench.bounds(pk, 2**30, 243.5 * 2**30, 0.0197, bench.DIVIDE_RECIP, 8)
    assert b["bound"] == "alu"
    assert abs(b["alu_frac"] - 243.5 * 2**30 / 5 / 0.0197 / 1e9 / 3500.0) < 1e-4
    assert b["frac"] == max(b["alu_frac"], b["fp64_frac"], b["hbm_frac"])
    # e = 3 (48 slots): 120 G outputs/s -> the reciprocal step on the FP64 pipe binds
    b = bench.bounds(pk, 120e9, 48 * 120e9, 1.0, bench.DIVIDE_RECIP, 16)
    assert b["bound"] == "fp64" and abs(b["fp64_frac"] - 0.75) < 1e-9
    # the integer route has no FP64 bound; the hybrid route puts 3 of 4 outputs on it
    assert bench.bounds(pk, 120e9, 48 * 120e9, 1.0, bench.DIVIDE_INT, 16)["fp64_frac"] is None
    h = bench.bounds(pk, 120e9, 48 * 120e9, 1.0, bench.DIVIDE_HYBRID, 16)
    assert abs(h["fp64_frac"] - 0.75 * 0.75) < 1e-9
    # IEEE division: division and conversion rates in series
    f = bench.bounds(pk, 10e9, 0, 1.0, bench.DIVIDE_FP64, 0)
    assert abs(f["fp64_frac"] - 10 * (1 / 70 + 1 / 300)) < 1e-4
    # nothing stored: no HBM work
    assert f["hbm_frac"] == 0.0


def test_cpu_oracle_forms():
    """The oracle timed beside the plain, batched and split forms: a positive rate on a
    bounded sample of each form's own workload, with the cores it used."""
    for name, k in (("plain_1x1e6", 1), ("batched_1e5_lognormal", 2000),
                    ("split_interleaved", 4096)):
        r = bench.cpu_oracle_form(name, target_s=0.05)
        assert r["kind"] == "oracle" and r["unit"] == bench.UNIT and r["value"] > 0
        assert r["cores"] == (1 if k == 1 else min(k, oracle.max_threads()))
        assert r["sample"].startswith(f"{k} instance")
