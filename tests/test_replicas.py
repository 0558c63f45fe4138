"""The multi-GPU form is replicas (every rank renders its own workload; no
step exchanges data). Its host logic runs here as two gloo ranks on the CPU:
the job time is the slowest rank's, the job throughput sums the ranks' units,
only rank 0 runs the CPU reference arm, and views that exceed one batch's
instance limit are split into consecutive batches."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        worst = bench.reduce_max(ms, world, "cpu")
        out.put((rank, worst, bench.job_throughput(50, world, worst)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [w for _, w, _ in res] == [20.0, 20.0]
    # 2 ranks x 50 frames in 20 ms
    assert all(abs(v - 5000.0) < 1e-9 for _, _, v in res)


def test_single_rank_needs_no_process_group():
    assert bench.reduce_max(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(10, 1, 100.0) == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        gpus, steps, warmup = 2, 1, 0
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_views_are_split_under_the_instance_limit():
    assert bench._chunks([5, 5, 5], 100) == [[0, 1, 2]]
    assert bench._chunks([60, 50, 30, 80], 100) == [[0], [1, 2], [3]]
    assert bench._chunks([150, 10], 100) == [[0], [1]]


def test_step_time_summary():
    d = bench.dist_summary([3.0, 1.0, 2.0, 10.0])
    assert d == {"n": 4, "median": 2.5, "mean": 4.0, "min": 1.0, "max": 10.0}
