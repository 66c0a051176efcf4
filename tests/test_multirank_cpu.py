"""Multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2).

Every rank holds a full replica of the index and searches its own query shard
(weak scaling, no data-path collective): the rows must be identical on all
ranks, the query shards distinct and deterministic, the job time the slowest
rank's (all-reduce MAX) and the job rate all ranks' queries over that time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    workload = "ivf_n1m_d960_nlist4096"
    nlist = 16
    n = 2000
    nq = 64
    scale = 1.0


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        cfg, X, Q, P = bench.make_workload(_Args(), rank)
        digest = torch.tensor([float(np.float64(X).sum()), float(np.float64(Q).sum()), float(np.float64(P).sum())],
                              dtype=torch.float64)
        allx = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allx, digest)
        ms = 10.0 + 5.0 * rank                                   # this rank's time
        job_ms = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.job_rate(len(Q), world, job_ms / 1e3)
        out[rank] = (allx[0].tolist(), allx[1].tolist(), job_ms, rate, len(Q))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (x0, x1, ms0, rate0, nq0), (y0, y1, ms1, rate1, nq1) = res[0], res[1]
    assert x0 == y0 and x1 == y1                     # both ranks saw the same gathered digests
    assert x0[0] == x1[0] and x0[2] == x1[2]         # identical rows and rotation on every rank
    assert x0[1] != x1[1]                            # distinct query shards
    assert ms0 == ms1 == 15.0                        # the slowest rank's time, on every rank
    assert rate0 == rate1 == pytest.approx(nq0 * world / 0.015)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(100, 1, 0.5) == 200.0
