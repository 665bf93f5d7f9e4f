"""The multi-process (torchrun) path of the benchmark on CPU with gloo, world size 2:
each rank runs its own replica with its own seed (the single graph does not shard, so
there is no collective on the data path), and the job's throughput is all ranks'
updates over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2202_04110_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # replica seed = rank: different inputs, same structure
    p = W.ising_grid(8, 8, seed=rank, n_iters=1)
    local_ms = 10.0 * (rank + 1)
    ms, value = bench.aggregate_ranks(dist, local_ms, updates_per_rank=1e6)
    sig = torch.tensor([float(abs(p.evidence).sum())], dtype=torch.float64)
    gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, sig)
    out[rank] = (ms, value, [float(x) for x in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        ms, value, sigs = out[r]
        assert ms == 20.0                        # the slowest rank's time
        assert abs(value - 2 * 1e6 / 0.020) < 1  # all ranks' updates over it
        assert sigs[0] != sigs[1]                # replicas draw different inputs
