"""Host logic of the multi-GPU benchmark (replicas, no collective in the data
path): the timed region's length is the slowest rank's, and the whole-job
value counts every replica.  Two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0 + 5.0 * rank, 3.0 - rank]   # rank 1 is slower in the first value, faster in the second
        out[rank] = bench.max_over_ranks(ms, device="cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == out[1] == [15.0, 3.0]


def test_job_value_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench

    one = bench.job_mlups(1, 2_097_152, 3000, 241.5)
    assert bench.job_mlups(4, 2_097_152, 3000, 241.5) == pytest.approx(4 * one)
    assert one == pytest.approx(2_097_152 * 3000 / 0.2415 / 1e6)
