"""Cluster-sharded search on two CPU ranks (gloo): the lists of one index are
split over the ranks, each rank searches its own lists with the FP64 oracle,
and the orchestration of paper_2409_09913_gb300.sharded (exchange of the
ranks' top-k' candidates, merge, exact re-rank of the merged candidates where
their rows live, final merge) must return exactly the single index's answer
(Section 4.1 search with the Eq. 3.3 estimator, exact re-rank of the top-k')."""
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

N, D, B, NLIST, NQ, K, KP, NPROBE = 3000, 64, 4, 12, 40, 5, 20, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    import synthetic as S
    X, lab = S.mixture(N, D, NLIST, 21, scale="aniso")
    Q, _ = S.mixture(NQ, D, NLIST, 22, comp_seed=21, scale="aniso")
    P = S.random_orthogonal(D, 23)
    return X, lab.astype(np.int32), Q, P


class OracleShard:
    """The FP64 oracle as the arithmetic of one rank (values in FP64)."""

    device = "cpu"

    def __init__(self, ox, Xr, nprobe, metric):
        self.ox, self.Xr, self.nprobe, self.metric = ox, Xr, nprobe, metric

    def search(self, Q, kp):
        import oracle
        r = oracle.search(self.ox, Q.numpy(), kp, kprime=kp, nprobe=self.nprobe, metric=self.metric)
        return torch.from_numpy(r["cand_ids"]), torch.from_numpy(r["cand_est"])

    def merge(self, ids, vals, k):
        ids, vals = ids.numpy(), vals.numpy()
        out_i = np.full((len(ids), k), -1, np.int64)
        out_v = np.full((len(ids), k), np.inf if self.metric == "l2" else -np.inf)
        for i in range(len(ids)):
            ok = ids[i] >= 0
            c, v = ids[i][ok], vals[i][ok]
            o = np.lexsort((c, v if self.metric == "l2" else -v))[:k]
            out_i[i, :len(o)], out_v[i, :len(o)] = c[o], v[o]
        return torch.from_numpy(out_i), torch.from_numpy(out_v)

    def rerank(self, Q, local_ids, k):
        import oracle
        i, v = oracle.rerank(self.Xr, Q.numpy(), local_ids.numpy(), k, metric=self.metric)
        return torch.from_numpy(i), torch.from_numpy(v)


def _rank_main(rank, world, port, metric, out):
    import oracle
    from paper_2409_09913_gb300 import sharded
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        X, lab, Q, P = _data()
        C = oracle.centroids(X, lab, NLIST)
        owner = sharded.partition_lists(np.bincount(lab, minlength=NLIST), world)
        rows = sharded.shard_rows(lab, owner, rank)
        ox = oracle.build_index(X[rows], P, lab[rows], NLIST, B, centroids_in=C)   # this rank's lists only
        be = OracleShard(ox, X[rows], NPROBE, metric)
        ids, vals = sharded.sharded_search(be, torch.from_numpy(Q.astype(np.float64)), K, KP,
                                           torch.from_numpy(rows), N)
        out[rank] = (ids.numpy(), vals.numpy(), len(rows))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_two_rank_sharded_search_equals_single_index(metric):
    import oracle
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, metric, out), nprocs=world, join=True)
        res = dict(out)
    X, lab, Q, P = _data()
    ref = oracle.search(oracle.build_index(X, P, lab, NLIST, B), Q, K, kprime=KP, nprobe=NPROBE, metric=metric)
    (i0, v0, n0), (i1, v1, n1) = res[0], res[1]
    assert n0 + n1 == N and n0 > 0 and n1 > 0                # every row on exactly one rank
    np.testing.assert_array_equal(i0, i1)                       # every rank ends with the same answer
    np.testing.assert_array_equal(i0, ref["ids"])               # ... the single index's
    np.testing.assert_allclose(v0, ref["dists"], rtol=1e-12)


def test_partition_lists_balances_rows():
    from paper_2409_09913_gb300 import sharded
    sizes = np.array([50, 10, 40, 30, 30, 20, 0])
    owner = sharded.partition_lists(sizes, 3)
    load = np.bincount(owner, weights=sizes, minlength=3)
    assert owner[0] == 0 and owner[2] == 1 and owner[3] == 2    # largest first, onto the emptiest rank
    assert load.max() - load.min() <= sizes.max()
    assert sorted(sharded.shard_rows(np.array([0, 2, 3, 0, 6]), owner, 0).tolist()) == [0, 3] + \
        ([4] if owner[6] == 0 else [])
