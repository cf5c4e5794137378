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


def test_traffic_record_matches_the_smoother_source():
    """The benchmark's DRAM-traffic figure is tied to a hash of the finest-level
    smoother's source (both headers of its body, the kernel, its launcher and the
    block-size rule).  The three definitions must still be found, and the committed
    record must carry the current hash, else the benchmark reports no traffic."""
    import json
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_1303_0008_gb300", "csrc", "mg_fp64.cu")
    text = open(csrc).read()
    for head in ("__global__ void __launch_bounds__(256) k_smooth_colour64(",
                 "int tpb_for(long long items)", "void launch_smooth64("):
        part = bench._definition(text, head)
        assert part.startswith(head) and part.rstrip().endswith("}")
    rec = json.load(open(os.path.join(root, "profiles", "traffic.json")))["k_smooth_colour64"]
    assert rec["source_hash"] == bench.kernel_source_hash()
    assert bench.traffic_per_launch("k_smooth_colour64") == rec["bytes_per_launch_full_size"] > 0
