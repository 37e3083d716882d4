"""Multi-GPU split of the batched form (CPU): independent graphs are assigned to
ranks by a greedy size balance, each rank runs its own set with no data-path
collective, and the whole-job figures are the updates of all ranks over the
slowest rank's time.  Two gloo ranks stand in for two GPUs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    return bench


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_shard_is_a_balanced_partition(parts):
    bench = _bench()
    rng = np.random.default_rng(parts)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(1e3), np.log(1e5), size=512))]
    sh = bench.shard_graphs(sizes, parts)
    assert len(sh) == parts
    flat = sorted(i for s in sh for i in s)
    assert flat == list(range(len(sizes)))  # every graph exactly once
    loads = [sum(sizes[i] for i in s) for s in sh]
    # greedy list scheduling in decreasing size: no part exceeds another by more than its smallest graph's share
    assert max(loads) - min(loads) <= max(sizes)
    assert bench.shard_graphs(sizes, parts) == sh  # deterministic


def test_shard_small_cases():
    bench = _bench()
    assert bench.shard_graphs([5, 3, 3, 2, 2, 1], 2) == [[0, 3, 5], [1, 2, 4]]
    assert bench.shard_graphs([7], 3) == [[0], [], []]
    assert bench.shard_graphs([], 2) == [[], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, sizes, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = bench.shard_graphs(sizes, world)[rank]
    # this rank "processes" its graphs: updates = sum of their sizes, 1 s per 1000 updates
    upd = float(sum(sizes[i] for i in mine))
    total, slowest = bench.whole_job(dist, upd, upd / 1000.0, "cpu")
    out[rank] = (mine, total, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_batched_shards_over_two_gloo_ranks():
    world = 2
    sizes = [900, 40, 300, 300, 250, 10, 600, 75]
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, sizes, out), nprocs=world, join=True)
        res = dict(out)
    mine0, mine1 = res[0][0], res[1][0]
    assert sorted(mine0 + mine1) == list(range(len(sizes))) and not set(mine0) & set(mine1)
    loads = [sum(sizes[i] for i in res[r][0]) for r in range(world)]
    for r in range(world):
        assert res[r][1] == float(sum(sizes))  # every rank's updates
        assert res[r][2] == max(loads) / 1000.0  # the slowest rank's time
