"""The benchmark's rank aggregation (max of the timed duration, sum of the solves)
with two gloo ranks on the CPU: independent solves shard across ranks with no
collective on the data path, only these two reductions."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    n = bench.sum_over_ranks(6.0)
    assert bench.world()[:2] == (rank, world)
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 12.0)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5 and bench.sum_over_ranks(6.0) == 6.0
