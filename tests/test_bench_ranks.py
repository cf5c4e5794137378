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


@pytest.mark.parametrize("kernel", ["k_smooth_colour64", "k_smooth_colour32_n", "k_half32",
                                    "k_smooth_slab32"])
def test_traffic_record_matches_the_smoother_source(kernel):
    """The benchmark's DRAM-traffic figures are tied to a hash of each roofline
    kernel's source (the headers of its body, the kernel and its launcher).  The
    definitions must still be found, and the committed record must carry the current
    hash, else the benchmark reports no traffic for that kernel."""
    import json
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    headers, unit, heads, *more = bench._KERNEL_SOURCES[kernel]
    csrc = os.path.join(root, "paper_1303_0008_gb300", "csrc")
    for f, head in [(unit, h) for h in heads] + list(more[0] if more else ()):
        part = bench._definition(open(os.path.join(csrc, f)).read(), head)
        assert part.startswith(head) and part.rstrip().endswith("}")
    rec = json.load(open(os.path.join(root, "profiles", "traffic.json")))[kernel]
    assert rec["source_hash"] == bench.kernel_source_hash(kernel)
    shapes = rec.get("by_tile32")
    if shapes:
        for tile, sub in shapes.items():
            full = bench.traffic_per_launch(kernel, 2 * rec["cells_per_launch"], tile32=int(tile))
            assert full == 2 * sub["bytes_per_launch"] > 0
        assert bench.traffic_per_launch(kernel, rec["cells_per_launch"], tile32=3) is None
    else:
        full = bench.traffic_per_launch(kernel, 2 * rec["cells_per_launch"])
        assert full == 2 * rec["bytes_per_launch"] > 0


def test_reference_arm_prints_one_line(capsys, monkeypatch):
    """The reference arm on a small grid: one JSON line with the contract's keys."""
    import json
    import bench
    monkeypatch.setattr(bench, "N", 32)
    monkeypatch.setattr(bench, "SAMPLE_CYCLES", 2)
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
