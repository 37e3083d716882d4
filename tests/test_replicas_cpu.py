"""The replicas path of bench.py (CPU, two gloo ranks): every rank runs its own
copy of the workload, with no data-path collective; the whole-job value is the
updates of all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r processed 1000 * (r + 1) updates in 2 + r seconds
    total, slowest = bench.whole_job(dist, 1000.0 * (rank + 1), 2.0 + rank, "cpu")
    out[rank] = (total, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (3000.0, 3.0)  # 1000 + 2000 updates, the slower rank's 3 s


def test_whole_job_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(None, 123.0, 4.5, "cpu") == (123.0, 4.5)
