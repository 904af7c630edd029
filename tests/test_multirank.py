"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): instance sharding
is disjoint per rank (weak scaling, no data-path collective) and the timing
reductions take the max / sum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import workload

    d = bench.Dist(backend_gpu=False)
    cfg = dict(workload.CONFIGS[bench.WORKLOAD])
    seeds = bench.rank_seeds(cfg, d.rank)
    elapsed = 1.0 + rank  # rank 1 is slower
    mx = d.max(elapsed)
    total = d.sum(float(len(seeds)))
    d.barrier()
    q.put((rank, seeds[:4].tolist(), seeds[-1].item(), mx, total))
    d.close()


def test_two_rank_sharding_and_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    import workload

    k = workload.CONFIGS["bulk_1024x2^20"]["instances"]
    all_seeds = workload.instance_seeds(workload.CONFIGS["bulk_1024x2^20"]["master"], 2 * k)
    for rank, head, last, mx, total in out:
        assert head == all_seeds[rank * k:rank * k + 4].tolist()
        assert last == int(all_seeds[(rank + 1) * k - 1])
        assert mx == 2.0  # max over ranks
        assert total == 2 * k  # work counted over all ranks
    assert not set(out[0][1]) & set(out[1][1])
    assert len(np.unique(all_seeds)) == 2 * k


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_contract_line(capsys):
    import json

    import bench

    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Gnumbers/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD


def test_bench_rejects_unknown_forms_before_any_work():
    import pytest

    import bench

    with pytest.raises(SystemExit, match="unknown forms"):
        bench.main(["--forms", "plain,bogus"])
    with pytest.raises(SystemExit, match="--parents"):
        bench.main(["--parents", "0"])
    assert set(bench.FORMS) >= {"plain", "batched", "served", "fused", "interleaved",
                                "split_full"}
