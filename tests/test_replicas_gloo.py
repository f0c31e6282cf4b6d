"""The multi-GPU path is replicas only (independent bundles per rank, no
collective on the data path). Its host logic runs here as two gloo ranks on
the CPU: every rank reports the slowest rank's time (element-wise MAX), the
whole-job throughput counts all ranks' units over that time, and the ranks'
bundles (seeded by rank) differ."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import bench
    import synth
    times = [10.0 + rank, 30.0 - 5 * rank, 7.5]
    got = bench.max_over_ranks(times, dist, device="cpu")
    rate = bench.aggregate_rate(20 * 3, world, got[0])
    sc = synth.make_scene("tiny", seed_offset=rank)
    fp = float(np.asarray(sc.images_store, np.float64).sum())
    dist.barrier()
    q.put((rank, got, rate, fp))
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, got, rate, _ in out:
        assert got == [11.0, 30.0, 7.5]  # element-wise max over the ranks
        assert abs(rate - 2 * 60 / (11.0 / 1e3)) < 1e-9
    assert out[0][3] != out[1][3]  # each rank solves its own bundle


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.aggregate_rate(100, 1, 50.0) == 2000.0
