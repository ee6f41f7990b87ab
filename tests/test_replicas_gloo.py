"""The multi-GPU path of bench.py (independent replicas, one chain per rank,
no data-path collective) on CPU: two gloo ranks check the per-rank seeds, the
max-over-ranks timing and the whole-job rate, and that the reference arm
runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank                    # rank 1 is the slow one
        t_max = bench.max_over_ranks(local_ms, dist, "cpu")
        # the reference arm prints on rank 0 only; other ranks return at once
        args = type("A", (), {"warmup": 0, "steps": 0, "bonds": 0})()
        out = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(out):
                bench.run_reference(args, rank, world)
        results[rank] = {"seed": bench.replica_seed(rank), "t_max": t_max,
                         "rate": bench.whole_job_rate(world, 4, t_max * 1e-3),
                         "ref_out": out.getvalue()}
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    port = _free_port()
    with mp.Manager() as manager:
        results = manager.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert set(res) == {0, 1}
    assert res[0]["seed"] != res[1]["seed"]                 # each rank evolves its own chain
    assert res[0]["t_max"] == res[1]["t_max"] == 150.0      # the slowest rank sets the time
    assert abs(res[0]["rate"] - world * 4 / 0.150) < 1e-9   # all ranks' steps over that time
    assert res[1]["ref_out"] == ""


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 3, 1.5) == 2.0
