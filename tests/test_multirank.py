"""The N > 1 bench path on CPU: two gloo ranks, each with its own share of independent problems
(no exchange on the data path), the job's time as the maximum over ranks and the solves as
the sum over ranks; each rank runs the oracle on its own small problem."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, out):
    import torch.distributed as dist
    import oracle.rqi_pcgtls as O
    from paper_2305_19028_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ids = bench._shard_ids(rank, 3)
        # each rank's own problem (the dense workload uses seed = rank)
        p = synth.dense_problem(60, 8, d_lo=1e-2, noise=1e-6, seed=rank)
        x, s, _ = O.rqi_pcgtls(p.A, p.b, tol=1e-12, max_rqi=10)
        ok = int(np.isfinite(s) and s > 0)
        t_max = bench._barrier_max(10.0 + rank, ws)
        total = bench._total(ok, ws)
        out.put((rank, ids, s, t_max, total))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, ids0, s0, t0, n0), (r1, ids1, s1, t1, n1) = res
    assert (r0, r1) == (0, 1)
    assert ids0 == [0, 1, 2] and ids1 == [3, 4, 5]          # disjoint shares, no overlap
    assert s0 != s1                                          # different problems per rank
    assert t0 == t1 == 11.0                                  # max over ranks
    assert n0 == n1 == 2.0                                   # sum over ranks


def test_single_rank_is_identity():
    assert bench._barrier_max(3.5, 1) == 3.5
    assert bench._total(7, 1) == 7
    assert bench._shard_ids(0, 4) == [0, 1, 2, 3]
