"""The bench's multi-rank path on the host: two gloo ranks (world size 2, 127.0.0.1) run the
rendezvous, the max-over-ranks timing rule and the whole-job value of bench.py, and the reference
arm's ranks other than 0 leave without work.  Replicas only: no data-path collective exists."""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws = bench.dist_setup()
    assert (r, ws) == (rank, world) and dist.get_backend() == "gloo"
    again = bench.dist_setup()  # idempotent: the reference arm calls it too
    assert again[1:] == (rank, world)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    value = bench.job_value(1000.0, ws, slowest)
    ref = None
    if rank != 0:
        ref = bench.run_reference(argparse.Namespace(gpus=world, steps=1, warmup=0, impl="reference",
                                                     alpha=0.5, N=4095, M=4096, rtol=1e-8))
    dist.barrier()
    out[rank] = (slowest, value, ref)
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    # both ranks see the slowest time (rank 1: 15 s) and the whole-job value 2 x 1000 / 15
    for r in (0, 1):
        assert res[r][0] == 15.0
        assert abs(res[r][1] - 2000.0 / 15.0) < 1e-12
    assert res[1][2] is None  # the reference arm's rank 1 returns without work
