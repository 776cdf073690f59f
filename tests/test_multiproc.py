"""The N > 1 benchmark runs independent replicas (one solve per rank, own
seed, no data-path collective) and reduces only the timing: value = attempts
of all ranks / max time over ranks.  Checked here with two gloo ranks on the
CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local, att_local = (2.0, 100.0) if rank == 0 else (3.0, 250.0)
    value, t_max, att = bench.aggregate_replicas(t_local, att_local, world, device="cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(7, rank))
    out[rank] = (value, t_max, att, tuple(seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replicas():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, t_max, att, seeds = res[rank]
        assert t_max == 3.0 and att == 350.0 and value == pytest.approx(350.0 / 3.0)
        assert seeds[0] != seeds[1]                     # independent replicas
