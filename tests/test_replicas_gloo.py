"""The multi-GPU path is independent replicas: the timing aggregation
(barrier, maximum of the elapsed times over ranks, whole-job throughput) on a
world-size-2 gloo process group on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_1608_06345_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert replicas.world() == (world, rank, rank)
    replicas.barrier()
    elapsed = [2.0, 5.0][rank]
    m = replicas.max_over_ranks(elapsed)
    out.put((rank, m, replicas.job_throughput(100.0, m, world)))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.0, 5.0]       # every rank sees the slowest
    assert [r[2] for r in res] == [40.0, 40.0]     # 2 x 100 units / 5 s


def test_single_process_needs_no_group():
    from paper_1608_06345_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10, 2.0, 1) == 5.0
