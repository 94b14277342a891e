"""The multi-rank path of bench.py (independent replicas, barrier and max-over-ranks timing)
with world size 2 over gloo on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    w, r, loc = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    v = bench.max_over_ranks(w, float(rank + 1) * 1.5)
    out[rank] = v
    dist.destroy_process_group()


def test_max_over_ranks_world2_gloo():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == 3.0 and out[1] == 3.0
