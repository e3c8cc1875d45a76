"""Replica aggregation of bench.py across ranks (gloo, world size 2, CPU):
the job's time is the slowest rank's, its bytes the sum over ranks."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, kms, kb = bench.aggregate_ranks(10.0 + rank, 2.0 * (rank + 1), 1e9 * (rank + 1), "cpu")
    out[rank] = torch.tensor([ms, kms, kb], dtype=torch.float64)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        ms, kms, kb = out[r].tolist()
        assert ms == 11.0 and kms == 4.0 and kb == 3e9
