"""The bench's multi-rank path on CPU (gloo, world size 2): per-rank
workloads (weak scaling, no data-path collective), whole-job aggregation
(points summed, step times the maximum over the ranks), and the reference
leg's rank-0-only report."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        res = bench.aggregate_over_ranks(1000.0 + rank, 2.0 + 3 * rank, 5.0 - rank, world, "cpu")
        out[rank] = (res, bench.rank_seed(7, rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate_and_shard():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        got = dict(out)
    for r in range(world):
        (pts, ms, e2e), seed = got[r]
        assert pts == 2001.0          # work of both ranks
        assert ms == 5.0 and e2e == 5.0  # the slowest rank's times
        assert seed == 7 + r          # each rank its own pair
    assert got[0][1] != got[1][1]


def test_single_rank_passthrough_and_reference_rank1_is_silent(capsys):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(5.0, 1.0, 2.0, 1, "cpu") == (5.0, 1.0, 2.0)

    class A:
        steps, warmup, gpus, seed = 1, 0, 2, 0
    assert bench.reference_main(A(), 1, 2) == 0  # rank 1: no work, no output
    assert capsys.readouterr().out == ""
