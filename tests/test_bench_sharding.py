"""Host-side logic of the multi-rank benchmark, on CPU with gloo (world 2):
row sharding covers every row once, and the reported time is the max over
ranks while the work is the sum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_shard_rows_partition():
    for world in (1, 2, 3, 8):
        rows = [k for r in range(world) for k in bench.shard_rows(100, world, r)]
        assert sorted(rows) == list(range(100))
        assert bench.shard_rows(100, world, 0)[0] == 99  # rank 0 takes the costliest row


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    k = bench.shard_rows(100, world, rank)[0]
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    g = torch.tensor([2.0 * 12 * k], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(g, op=dist.ReduceOp.SUM)
    out[rank] = (k, float(t.item()), float(g.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == 99 and res[1][0] == 98
    for r in (0, 1):
        assert res[r][1] == 2.0                      # max over ranks
        assert res[r][2] == 2.0 * 12 * (99 + 98)     # G-steps summed over ranks
