"""The multi-rank path of bench.py (independent replicas, one per rank) on
CPU: two gloo ranks agree on the slowest rank's time and report every
rank's cell updates over it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench._dist()[:2] == (rank, world)
    ms, v = bench.replica_throughput(10.0 * (rank + 1), 1000, 50, dist, "cpu")
    out[rank] = (ms, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, v = res[0]
    assert ms == 20.0
    assert v == pytest.approx(2 * 1000 * 50 / 0.020 / 1e6)


def test_single_rank_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, v = bench.replica_throughput(4.0, 2000, 10)
    assert ms == 4.0 and v == pytest.approx(2000 * 10 / 0.004 / 1e6)


def test_algorithmic_bytes_of_the_roofline():
    """The bench's byte counts: every population read and written once and
    rho, phi, psi written and read once is 480 B per FP32 cell update (the
    figure of the lattice update); 16-bit storage keeps the two rest
    populations in FP32 (118 B of populations, 260 B per update).  The tau
    = 1 kernels add j (12 B each way)."""
    import bench
    assert bench.pop_bytes(4) == 228 and bench.step_bytes(4) == 480
    assert bench.pop_bytes(2) == 118 and bench.step_bytes(2) == 260
    assert bench.kernel_bytes(4) == {"k_moments": 252, "k_collide": 256}
    assert bench.kernel_bytes(4, t1=False) == {"k_moments": 240, "k_collide": 472}
    assert bench.kernel_bytes(2) == {"k_moments": 142, "k_collide": 146}
