"""Host-side logic of bench.py without a GPU: max-over-ranks timing and
sum-over-ranks work across two gloo ranks, and the reference (oracle) arm."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds, pairs = bench.aggregate(1.0 + rank, 10.0 * (rank + 1))
    bench.barrier()
    out[rank] = (seconds, pairs)
    dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sum_of_work_over_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        assert res[rank] == (2.0, 30.0)


def test_aggregate_without_process_group_is_identity():
    assert bench.aggregate(3.5, 7.0) == (3.5, 7.0)


def test_reference_arm_prints_one_json_line(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--workload", "tiny", "--steps", "1",
                       "--warmup", "0"]) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["unit"] == "pairs/s" and rec["higher_is_better"] is True
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_non_zero_rank_does_nothing(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    assert bench.main(["--impl", "reference", "--workload", "tiny", "--steps", "1",
                       "--warmup", "0"]) == 0
    assert capsys.readouterr().out.strip() == ""
