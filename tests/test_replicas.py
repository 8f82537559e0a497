"""The N > 1 path of bench.py on the CPU: two gloo ranks run the replica
aggregation (max over ranks of the elapsed times, whole-job throughput), and
the reference arm does no work on ranks other than 0."""
import json
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    # each rank measured its own replica: rank 1 is slower on the first
    # timing, rank 0 on the second
    mine = (100.0 + 50.0 * rank, 200.0 - 30.0 * rank)
    dist.barrier()
    times, values = bench.replica_totals(dist, "cpu", mine, steps=10, world=world)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as fh:
        json.dump({"times": times, "values": values}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_replicas(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for g in got:
        assert g["times"] == [150.0, 200.0]                # max over ranks
        solves = 4 * 10 * 2                                 # 4 permutations x 10 steps x 2 ranks
        assert g["values"] == pytest.approx([solves / 0.150, solves / 0.200])


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    times, values = bench.replica_totals(None, "cpu", (250.0,), steps=5, world=1)
    assert times == [250.0] and values == pytest.approx([4 * 5 / 0.25])


def test_reference_arm_works_on_rank_0_only():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, 1, 2) is None          # returns at once, no oracle work
