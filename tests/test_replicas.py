"""The multi-GPU path on the CPU: two gloo ranks run the replica helpers the
benchmark uses on N GPUs (each rank its share of independent problems, the
slowest rank's time, the job's total work)."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    import torch.distributed as dist

    from paper_0704_2344_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard(list(range(11)), rank, world)
        slowest = replicas.max_over_ranks([1.0 + rank, 10.0 - rank])
        total = replicas.sum_over_ranks([len(mine)])
        replicas.barrier()
        queue.put((rank, mine, slowest, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, mine, slowest, total = queue.get(timeout=120)
            out[rank] = (mine, slowest, total)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    shares = [set(out[r][0]) for r in range(2)]
    assert shares[0].isdisjoint(shares[1]) and shares[0] | shares[1] == set(range(11))
    for r in range(2):
        assert out[r][1] == [2.0, 10.0]   # element-wise maximum over the ranks
        assert out[r][2] == [11.0]        # the whole job's work


def test_single_process_is_a_no_op():
    from paper_0704_2344_gb300 import replicas
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.max_over_ranks([3.0]) == [3.0]
    replicas.barrier()
