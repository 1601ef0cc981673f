"""The N > 1 path of the benchmark (independent replicas, one per GPU, no
collective on the data path): the cross-rank gather of per-rank stats and
the whole-job aggregate, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r did (r+1) million updates per step over 10 steps in (2 + r) ms per step
    vals = bench.replica_stats([10 * (rank + 1) * 1e6, 2.0 + rank, 1e8 * (rank + 1)], "cpu")
    value, ms, e2e = bench.aggregate_replicas(vals, 10)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([value, ms, e2e, *vals.ravel()]))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregate_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)                      # every rank sees the same gather
    value, ms, e2e = r0[:3]
    # 30 million updates in total over the slowest rank's 10 x 3 ms
    assert ms == 3.0
    assert value == pytest.approx(30e6 / 30e-3, rel=1e-15)
    assert e2e == pytest.approx(3e8, rel=1e-15)
    assert np.array_equal(r0[3:].reshape(world, 3), [[10e6, 2.0, 1e8], [20e6, 3.0, 2e8]])
