"""Host-side logic of bench.py without a GPU: max-over-ranks timing and
sum-over-ranks work across two gloo ranks, the reference (oracle) arm, the
roofline arithmetic, the DRAM traffic records and the stage schedules."""
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


def test_roofline_takes_the_slower_call_at_the_finest_level(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    fwd = {0: 0.30, 1: 0.31, 2: 0.35}
    adj = {0: 0.33, 1: 0.34, 2: 0.40}
    counts = [100_000, 99_000, 98_000]
    h = 1.5 / 40.0  # mm per cell at 40 MHz
    r = bench.roofline(fwd, adj, counts, 512, {"sm_mhz": 2000.0}, 3.35 * h, h, None)
    assert r["kernel"] == "adjoint call at the finest level"
    assert r["pairs_per_launch"] == 98_000 * 512 and r["ms_per_launch"] == 0.40
    # 156 operations per pair, 3 per ramp cell past the first, 2 for the ends
    assert r["ops_per_pair"] == pytest.approx(156 + 3 * (6.7 - 1) + 2)
    assert r["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e9)
    achieved = 98_000 * 512 * r["ops_per_pair"] / 0.40e-3 / 1e9
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / r["peak"])
    # the forward's count when its call is the slower one
    r = bench.roofline({2: 0.5}, {2: 0.4}, [0, 0, 1000], 8, {"sm_mhz": 2070.0}, 0.1, h, None)
    assert r["kernel"] == "forward call at the finest level"
    assert r["ops_per_pair"] == bench.FWD_OPS_PER_PAIR


def test_traffic_record_holds_only_for_the_measured_sources(monkeypatch):
    rec = dict(bench.NCU_TRAFFIC["adjoint"])
    assert bench._traffic("adjoint") in (None, rec["bytes"])
    import hashlib

    m = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(bench.ROOT, src), "rb") as f:
            m.update(f.read())
    good = dict(rec, sha256=m.hexdigest()[:16])
    monkeypatch.setitem(bench.NCU_TRAFFIC, "adjoint", good)
    assert bench._traffic("adjoint") == rec["bytes"]
    monkeypatch.setitem(bench.NCU_TRAFFIC, "adjoint", dict(good, sha256="0" * 16))
    assert bench._traffic("adjoint") is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "adjoint", dict(good, bytes=None))
    assert bench._traffic("adjoint") is None


def test_stage_schedules():
    """Coarse stage (p0 and R) 40 iterations per level coarse to fine, then
    the fine stage (all components) 30 per coarser level and the rest at the
    finest; the ablation stays at the finest level throughout."""
    seg = 10
    it = bench.pro_segments(3, seg)
    head = [next(it) for _ in range(12 + 6 + 3)]
    assert head[:12] == [(0, 3)] * 4 + [(1, 3)] * 4 + [(2, 3)] * 4
    assert head[12:18] == [(0, 7)] * 3 + [(1, 7)] * 3
    assert head[18:] == [(2, 7)] * 3
    it = bench.flat_segments(3, seg)
    head = [next(it) for _ in range(15)]
    assert head == [(2, 3)] * 12 + [(2, 7)] * 3
