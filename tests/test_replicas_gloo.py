"""The N > 1 host path of bench.py on CPU: two gloo ranks stand in for two GPUs.

With one GPU per box the benchmark runs replicas (each rank its own copy of the
workload); what crosses ranks is the barrier and the maximum of the timings.  These
tests run that logic under torch.distributed with the gloo backend, world size 2.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "measured" these step times (ms): the job's times are the per-entry maxima
        local = [10.0 + rank, 5.0 - rank, 7.0 + 3.0 * rank]
        got = bench.max_over_ranks(local, world)
        dist.barrier()
        # rank 0's reference arm would time the CPU oracle; only the others' is checked here
        ref_line = (bench.run_reference(bench.parse(["--impl", "reference"]), rank, world)
                    if rank else None)
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"max": got, "reference_line": ref_line}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["max"] == [11.0, 5.0, 10.0]
    # the reference arm runs on rank 0 alone; the other ranks do no work and print nothing
    assert res[1]["reference_line"] is None


def test_whole_job_rate_counts_every_replica():
    # 2 replicas x 100 units x 3 steps in 0.5 s
    assert bench.job_rate(100, 3, 500.0, 2) == pytest.approx(1200.0)
    assert bench.job_rate(100, 3, 500.0, 1) == pytest.approx(600.0)
    assert bench.max_over_ranks([1, 2.5], 1) == [1.0, 2.5]


def test_reference_arm_prints_nothing_off_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()
    assert capsys.readouterr().out == ""
