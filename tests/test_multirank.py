"""The multi-GPU path of the benchmark on CPU: two gloo ranks.

The path shards by replication: every rank evaluates its own seeded copy of
the workload with no collective on the data path; the only communication is
the barrier and the max-over-ranks reduction of the step time.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(local_ms, dist, "cpu")
        dist.barrier()
        out[rank] = t
        out[world + rank] = bench.job_throughput(world, 1e9, t * 1e-3)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Array("d", 2 * world)
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    assert list(out[:world]) == [15.0, 15.0]
    # 2 ranks x 1e9 units each in 15 ms: 2 / 0.015 G units/s, same on both ranks
    assert np.allclose(out[world:], 2.0 / 0.015)


def test_single_process_helpers():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 2e9, 2.0) == 1.0


def test_replicas_get_distinct_seeded_workloads():
    w0 = bench.workload(17, 10, rank=0)
    w1 = bench.workload(17, 10, rank=1)
    assert not np.array_equal(w0.f, w1.f)
    assert np.array_equal(w0.f, bench.workload(17, 10, rank=0).f)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        m, probes, warmup, steps = 17, 10, 1, 1

    assert bench.run_reference(A) == 0


def test_traffic_is_reported_only_for_the_profiled_sources(monkeypatch):
    """bench.py takes the pair kernel's DRAM traffic from the committed ncu
    summary only while the hash of the kernel sources matches the one the
    summary was taken on; any other source state reports null."""
    import bench
    committed = bench.traffic_from_profile()
    text = open(os.path.join(bench.ROOT, "profiles", "pair32_dram_traffic.txt")).read()
    recorded = [l.split(":", 1)[1].strip() for l in text.splitlines()
                if l.startswith("source_sha256:")][0]
    monkeypatch.setattr(bench, "pair32_source_hash", lambda: recorded)
    assert bench.traffic_from_profile() == float(
        [l.split(":", 1)[1] for l in text.splitlines() if l.startswith("dram_bytes_per_launch")][0])
    monkeypatch.setattr(bench, "pair32_source_hash", lambda: "0" * 64)
    assert bench.traffic_from_profile() is None
    assert committed is None or committed > 0


def test_clock_summary_of_nvidia_smi_lines():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
             "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",
             "garbled\n"]
    c = bench.clock_summary(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    hot = lines[:1] + ["0, 1500, 2070, 800.0, 0x48, Active, Active, Not Active, Not Active\n"]
    assert bench.clock_summary(hot)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.clock_summary(hot)["sm_mhz"] == 1785.0
    assert bench.clock_summary([]) is None and bench.clock_summary(["x, y\n"]) is None


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the keys of the benchmark contract, its own CPU-baseline record and a
    host-only e2e record (no device copies)."""
    import json

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        m, probes, warmup, steps = 17, 10, 0, 1

    bench.run_reference(A)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
