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
