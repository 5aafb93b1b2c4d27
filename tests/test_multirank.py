"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1. Every rank refines its own copy of
the same seeded workload (replicas, no collective on the data path); the only collectives are the
barrier and the max over ranks of the timed region, and the whole-job rate counts every rank's
units against the slowest rank."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_1809_06047_gb300 import synth
        m = synth.workload("cc_torus16_L3")
        # each replica refines its own copy; results must agree bit for bit across ranks
        out = oracle.subdivide(m, 2, "cc", keep_all=False)[-1]
        digest = np.frombuffer(out["P"].tobytes(), dtype=np.uint8).astype(np.int64).sum()
        dist.barrier()
        ms_local = 10.0 * (rank + 1)                        # rank 1 is the slow one
        ms_max = bench.reduce_max(ms_local, dist, "cpu")
        rate = bench.whole_job_rate(out["F"], world, ms_max)
        import torch
        d = torch.tensor([int(digest), out["F"]], dtype=torch.int64)
        gathered = [torch.zeros_like(d) for _ in range(world)]
        dist.all_gather(gathered, d)
        q.put((rank, ms_max, rate, [g.tolist() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ms_max, rate, gathered in res:
        assert ms_max == 20.0                               # max over ranks, seen by both
        F = gathered[0][1]
        assert rate == pytest.approx(F * 2 / 0.020)         # both ranks' faces over the slowest time
        assert gathered[0] == gathered[1]                   # identical replicas
    assert res[0][3] == res[1][3]


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_rate(1000, 1, 500.0) == pytest.approx(2000.0)
    assert bench.percentile([5, 1, 4, 2, 3], 0.5) == 3
    assert bench.percentile(list(range(1, 101)), 0.99) == 99
    assert bench.percentile([], 0.5) is None
    a = bench.parse(["--gpus", "1", "--steps", "3", "--warmup", "3", "--no-serving"])
    assert a.steps == 3 and a.no_serving
