"""The multi-GPU form of the benchmark is replicas only (each rank solves its own problem,
no collective on the data path).  Its host logic -- max-over-ranks time, whole-job
throughput -- runs here on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [3.0, 5.0][rank]          # rank 1 is the slower replica
    total, value = bench.replica_aggregate(local, steps=4, world=world, dist=dist)
    dist.barrier()
    out[rank] = (total, value)
    dist.destroy_process_group()


def test_replicas_take_max_time_and_count_all_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        total, value = res[rank]
        assert total == 5.0
        assert value == pytest.approx(2 * 4 / 5.0)


def test_single_rank_needs_no_collective():
    assert bench.replica_aggregate(2.0, steps=3, world=1) == (2.0, 1.5)
