"""The benchmark's multi-rank path on the CPU: two gloo ranks (one process each, as torchrun
starts them) time different amounts of work; both must report the whole job's frames over the
slowest rank's time.  The analysis path shards by video with no data exchange, so this timing
reduction is the only collective of a multi-GPU run."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    barrier, max_over_ranks = bench.rank_reducers(world, "gloo")
    barrier()
    value, ms_per_step = bench.whole_job_rate(100.0 + 50.0 * rank, 10, 64, world, max_over_ranks)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{value} {ms_per_step}")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_whole_job(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    slowest_ms = 100.0 + 50.0 * (world - 1)
    for rank in range(world):
        value, ms_per_step = map(float, open(tmp_path / f"rank{rank}.txt").read().split())
        assert value == pytest.approx(world * 10 * 64 / (slowest_ms / 1000.0))
        assert ms_per_step == pytest.approx(slowest_ms / 10)


def test_single_rank_needs_no_process_group():
    import bench

    barrier, max_over_ranks = bench.rank_reducers(1)
    barrier()
    assert bench.whole_job_rate(200.0, 10, 64, 1, max_over_ranks) == (3200.0, 20.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"gpus": 2, "steps": 1, "warmup": 1})()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
