"""Cluster-sharded search with the library on the GPU: two shards of one
index (lists split by partition_lists, each shard built with the global
centroids) searched through paper_2409_09913_gb300.sharded with the library's
merge and re-rank, the exchange emulated between two host threads (the
shards' kernels never wait on each other), must return exactly the single
index's answer (Section 4.1: each owner's top-k' holds all of its members of
the global top-k')."""
import threading

import numpy as np
import pytest
import torch

import synthetic as S
from gpu_common import erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


class ThreadComm:
    """all_gather between host threads of one process (one per shard)."""

    def __init__(self, rank, world, shared):
        self.rank, self.world, self.sh = rank, world, shared

    def world_size(self):
        return self.world

    def all_gather(self, out, t):
        self.sh["slots"][self.rank] = t
        self.sh["bar"].wait()
        for r in range(self.world):
            out[r].copy_(self.sh["slots"][r])
        self.sh["bar"].wait()                    # every thread has read the slots


@pytest.mark.parametrize("precision,metric", [("fp32", "l2"), ("fp16", "l2"), ("fp32", "ip")])
def test_two_shards_equal_the_single_index(erq, precision, metric):
    from paper_2409_09913_gb300 import sharded
    N, D, B, nlist, nq, k, kp, nprobe = 20000, 128, 5, 32, 120, 10, 30, 6
    X, _ = S.mixture(N, D, 16, 5600, scale="aniso")
    assign = S.kmeans_assign(X, nlist, 4, 5601)
    P = S.random_orthogonal(D, 5602)
    Q, _ = S.mixture(nq, D, 16, 5603, comp_seed=5600, scale="aniso")
    gx = erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(assign))
    ref_i, ref_v = gx.search(to_dev(Q), k, rerank_k=kp, nprobe=nprobe, precision=precision, metric=metric)
    C = gx.export("centroids").to("cuda")
    owner = sharded.partition_lists(np.bincount(assign, minlength=nlist), 2)
    shards = []
    for r in range(2):
        rows = sharded.shard_rows(assign, owner, r)
        ix = erq.build_index(to_dev(X[rows]), to_dev(P), B, nlist, assign=to_dev(assign[rows]), centroids=C)
        shards.append((ix, torch.from_numpy(rows).to("cuda")))
    assert sum(len(g) for _, g in shards) == N
    shared = {"slots": [None, None], "bar": threading.Barrier(2)}
    out, errs = [None, None], []
    Qd = to_dev(Q)

    def run(r):
        try:
            be = sharded.ErqShard(shards[r][0], {"nprobe": nprobe, "precision": precision}, metric=metric)
            out[r] = sharded.sharded_search(be, Qd, k, kp, shards[r][1], N, comm=ThreadComm(r, 2, shared))
            torch.cuda.synchronize()
        except Exception as ex:                  # reported by the main thread
            errs.append(ex)
            shared["bar"].abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    (i0, v0), (i1, v1) = out
    assert torch.equal(i0, i1) and torch.equal(v0, v1)
    assert torch.equal(i0.cpu(), ref_i.cpu())
    np.testing.assert_array_equal(v0.cpu().numpy(), ref_v.cpu().numpy())
