"""The benchmark's multi-rank host logic on CPU (gloo, world size 2).

The path does not shard: under torchrun every rank solves its own replica and
the job's time is the slowest rank's, taken with one MAX all-reduce after the
timed region (NCCL on the GPUs; the same helper with a CPU tensor on gloo).
The reference arm runs on rank 0 only; the other ranks return without work
or output.
"""
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    import bench
    slowest = bench.max_over_ranks(10.0 + 3.0 * rank, ws, None)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}"), "w") as f:
        f.write(repr(slowest))
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got = [float((tmp_path / f"rank{r}").read_text()) for r in range(2)]
    assert got == [13.0, 13.0]


def test_single_rank_time_is_unchanged():
    import bench
    assert bench.max_over_ranks(7.5, 1, None) == 7.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = types.SimpleNamespace(warmup=3, steps=2, workload="precision", extra={}, gpus=2)
    assert bench.run_reference(args, None) is None
    assert capsys.readouterr().out == ""
