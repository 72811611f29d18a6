"""The N > 1 path of bench.py (independent replicas, one lattice per GPU, no
data-path collective) on CPU: two gloo ranks check the timing aggregation
(max over ranks, whole-job throughput) and that each replica's result is the
same FP64 oracle answer regardless of rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from synth import fields
    # each replica does its own (identical) unit of work
    dims = (4, 4, 4, 4)
    U = fields.su3_links(dims, workers=1)
    psi = fields.gaussian_spinor(dims)
    r = oracle.hop_block(0, oracle.restrict(psi, dims, 1), U, dims)
    local_seconds = 1.0 + rank  # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_seconds, "cpu")
    value = bench.replica_value(100.0, world, slowest)
    out[rank] = (slowest, value, float(np.linalg.norm(r)))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == out[1][1] == pytest.approx(100.0)
    assert out[0][2] == out[1][2]
