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


def _levels(fwd, adj, counts, M, mean_R, hs):
    return [{"mhz": 40.0 / (2 ** (len(hs) - 1 - k)), "h_mm": hs[k], "pairs": counts[k] * M,
             "mean_R_mm": mean_R[k], "forward_ms": fwd[k], "adjoint_ms": adj[k]}
            for k in range(len(hs))]


def test_roofline_counts_the_methods_operations_per_sample(monkeypatch):
    """forward 25 + 6 s, adjoint 40 + 8 s, both together 80 + 14 s operations
    per pair, s = 2 R / h + 1 at the live cloud's mean radius; the dominant
    kernel is the one with the larger time over the step, taken at its
    finest-level launch."""
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    h = 1.5 / 40.0  # mm per cell at 40 MHz
    hs = [4 * h, 2 * h, h]
    R = [0.125, 0.13, 0.14]
    counts = [100_000, 99_000, 98_000]
    lv = _levels([0.30, 0.31, 0.35], [0.33, 0.34, 0.40], counts, 512, R, hs)
    r = bench.roofline(lv, {"sm_mhz": 2000.0}, None)
    assert r["kernel"].startswith("adjoint at 40 MHz")
    assert r["pairs_per_launch"] == 98_000 * 512 and r["ms_per_launch"] == 0.40
    s = 2 * 0.14 / h + 1
    assert r["samples_per_pair"] == pytest.approx(s)
    assert r["ops_per_pair"] == pytest.approx(40 + 8 * s)
    assert r["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e9)
    achieved = 98_000 * 512 * (40 + 8 * s) / 0.40e-3 / 1e9
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / r["peak"])
    fa = r["per_level"][2]["forward+adjoint"]
    assert fa["pairs_per_s"] == pytest.approx(98_000 * 512 / 0.75e-3)
    assert fa["ceiling_pairs_per_s"] == pytest.approx(r["peak"] * 1e9 / (80 + 14 * s))
    s0 = 2 * 0.125 / (4 * h) + 1
    assert r["per_level"][0]["forward"]["ops_per_pair"] == pytest.approx(25 + 6 * s0)
    step_ops = sum(counts[k] * 512 * (80 + 14 * (2 * R[k] / hs[k] + 1)) for k in range(3))
    assert r["forward_adjoint_frac_step"] == pytest.approx(
        step_ops / (sum([0.30, 0.31, 0.35, 0.33, 0.34, 0.40]) * 1e-3) / 1e9 / r["peak"])
    # the forward when it takes longer over the step
    lv = _levels([0.5, 0.5, 0.5], [0.4, 0.4, 0.4], [1, 1, 1000], 8, R, hs)
    r = bench.roofline(lv, {"sm_mhz": 2070.0}, None)
    assert r["kernel"].startswith("forward")
    assert r["ops_per_pair"] == pytest.approx(25 + 6 * s)


def test_ncu_record_holds_only_for_the_measured_sources(monkeypatch):
    rec = dict(bench.NCU_RECORD["adjoint"])
    assert bench.ncu_record("adjoint") in ((None, None),
                                           (rec["bytes"], rec["thread_inst_per_pair"]))
    good = dict(rec, sha256=bench.sources_sha("adjoint"), bytes=1.5e6,
                thread_inst_per_pair=120.0)
    monkeypatch.setitem(bench.NCU_RECORD, "adjoint", good)
    assert bench.ncu_record("adjoint") == (1.5e6, 120.0)
    monkeypatch.setitem(bench.NCU_RECORD, "adjoint", dict(good, sha256="0" * 16))
    assert bench.ncu_record("adjoint") == (None, None)


def test_record_hash_follows_the_kernel_not_host_declarations(monkeypatch, tmp_path):
    """The ncu record's source hash changes with the kernel's file, with a
    #define of the shared header and with the header's device code, but not
    with a host declaration added to the header."""
    import shutil

    rec = bench.NCU_RECORD["adjoint"]
    for src in rec["sources"]:
        (tmp_path / src).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, src), tmp_path / src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.sources_sha("adjoint")
    hdr = tmp_path / [s for s in rec["sources"] if s.endswith(".cuh")][0]
    text = hdr.read_text()
    mark = bench.DEVICE_MARK.decode()
    i = text.index(mark)
    hdr.write_text(text[:i] + "int some_host_function(int);\n" + text[i:])
    assert bench.sources_sha("adjoint") == base
    hdr.write_text(text.replace("#define SBP_ADJ_MAX_SPLIT 8", "#define SBP_ADJ_MAX_SPLIT 16"))
    assert bench.sources_sha("adjoint") != base
    hdr.write_text(text + "// a device-side change\n")
    assert bench.sources_sha("adjoint") != base


def test_run_to_residual_interpolates_every_crossing(monkeypatch):
    """run_to_residual with a fake array whose segments take 1 ms of device
    time each and a residual falling 0.9, 0.6, 0.4, 0.25, 0.15: the target
    (0.2) and the looser targets (0.5, 0.3) are reached at the linear
    interpolation of their two neighbouring checkpoints."""
    torch = pytest.importorskip("torch")

    class FakeEvent:
        clock = [0.0]

        def __init__(self, enable_timing=True):
            self.t = None

        def record(self, stream=None):
            self.t = FakeEvent.clock[0]

        def elapsed_time(self, other):
            return other.t - self.t

    class FakeArr:
        def reconstruct(self, *args, **kwargs):
            FakeEvent.clock[0] += 1.0  # 1 ms per segment

    class FakeSb:
        KEEP_NEG = 0

        @staticmethod
        def Stage(*a):
            return a

        @staticmethod
        def GrowParams(**kw):
            return kw

    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    seq = iter([0.9, 0.6, 0.4, 0.25, 0.15])
    init = torch.zeros((5, 8))
    out = bench.run_to_residual(FakeSb, FakeArr(), None, None, init, 8,
                                iter([(0, 3)] * 10), True, 0.2, 10, 1000,
                                lambda balls, n: next(seq), also=(0.5, 0.3, 0.2))
    # checkpoints (ms, r): (1, .9) (2, .6) (3, .4) (4, .25) (5, .15)
    assert out["iterations"] == 50 and out["final_rel_residual"] == 0.15
    assert abs(out["seconds"] - (4.0 + (0.25 - 0.2) / (0.25 - 0.15)) * 1e-3) < 1e-12
    to = out["seconds_to"]
    assert abs(to["0.5"] - (2.0 + (0.6 - 0.5) / (0.6 - 0.4)) * 1e-3) < 1e-12
    assert abs(to["0.3"] - (3.0 + (0.4 - 0.3) / (0.4 - 0.25)) * 1e-3) < 1e-12
    assert abs(to["0.2"] - out["seconds"]) < 1e-15


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
