"""Multi-GPU runs are independent replicas (one solve stream per rank, no
data-path collective): the whole-job value is all ranks' units over the
slowest rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 5 + rank                  # ranks may process different amounts
    ms = 100.0 * (rank + 1)
    value, ms_max = bench.replica_throughput(dist, units, ms, "cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    total_units, slowest_ms = 5 + 6, 200.0
    for r in range(world):
        value, ms_max = res[r]
        assert ms_max == slowest_ms
        assert abs(value - total_units / (slowest_ms / 1e3)) < 1e-9


def test_replica_throughput_single_process():
    import bench
    value, ms = bench.replica_throughput(None, 4, 50.0, "cpu")
    assert value == 4 / 0.05 and ms == 50.0
