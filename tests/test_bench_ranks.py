"""Host logic of the benchmark's N > 1 path on CPU: independent replicas,
whole-job time = the slowest rank, work = the sum over ranks, and the
reference arm runs on rank 0 only.  Two gloo ranks, no GPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import json
    import sys

    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # rank r took (10 + r) ms and 3 + r seconds end to end, did 100 (r + 1) units
    slow, summed = bench.combine_ranks(dist, [10.0 + rank, 3.0 + rank], [100.0 * (rank + 1), 7.0], "cpu")
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slow": slow, "summed": summed}, f)


def test_two_gloo_ranks_combine_max_time_and_summed_work(tmp_path):
    import json

    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["slow"] == [11.0, 4.0]          # the slowest rank's times
        assert d["summed"] == [300.0, 14.0]      # work of both ranks


def test_single_rank_passes_figures_through():
    import bench
    assert bench.combine_ranks(None, [1.5, 2.0], [3.0], "cpu") == ([1.5, 2.0], [3.0])


def test_reference_arm_does_no_work_off_rank_0(monkeypatch, capsys):
    import types

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")
    monkeypatch.setattr(bench, "run_oracle", boom)
    assert bench.reference_arm(types.SimpleNamespace(steps=2, warmup=3, gpus=2)) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """The reference arm (the oracle on the host) prints one JSON line with
    the keys the benchmark contract asks of it (one short oracle step)."""
    import json
    import types

    import bench
    monkeypatch.setenv("RANK", "0")
    assert bench.reference_arm(types.SimpleNamespace(steps=1, warmup=0, gpus=1)) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_cpu_baseline_reports_one_and_all_cores(monkeypatch):
    """cpu_baseline runs the C2 sample and C1 in full, each on one thread and
    as one replica per host core, and reports the all-core C2 rate as value
    (oracle runs replaced by a stand-in that returns fixed timings)."""
    import bench
    calls = []

    def fake(sample, steps, copies=1):
        calls.append((sample["n"], steps, copies))
        return 100, 2.0, [[(1.0, 5)] * steps for _ in range(copies)]
    monkeypatch.setattr(bench, "run_oracle", fake)
    monkeypatch.setattr(bench, "host_cores", lambda: 4)
    cb = bench.cpu_baseline()
    assert sorted(calls) == sorted([(bench.REF_NX, 1, 1), (bench.REF_NX, 1, 4), (20, 10, 1), (20, 10, 4)])
    assert cb["cores"] == 4 and cb["kind"] == "oracle" and cb["host"]["nproc"] == 4
    assert cb["value"] == 4 * 100 * 5 / 2.0
    assert cb["single_thread_value"] == 100 * 5 / 2.0
    assert cb["runs"]["c1_full"]["all_cores"]["value"] == 4 * 100 * 50 / 2.0
