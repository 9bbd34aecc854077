"""Multi-process path of the benchmark on CPU (gloo, world size 2): the path has no exchange
between views, so N GPUs run N independent replicas; the job time is the slowest replica's
(max over ranks) and the throughput counts every replica's pixels."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    out[rank] = bench.max_over_ranks(ms, torch.device("cpu"), world)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_throughput():
    import bench
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 15.0
    # 2 replicas x 1 Mpix x 10 steps in 15 ms of the slowest replica
    assert abs(bench.whole_job_mpix(1_000_000, 2, 10, 15.0) - 2 * 1.0 * 10 / 0.015) < 1e-6
