"""Cluster-sharded search over several GPUs with one exchange step.

The IVF lists of one index (Section 4.1) are partitioned over the ranks of a
torch.distributed group, one rank per GPU.  Every rank holds the full
centroid set and P, the queries, and the rows, codes and factors of the lists
it owns only (an index built with the global centroids, so its codes, factors
and probe are the single index's).  A batch is searched in five steps:

1. probe and scan (every rank, erq_search without re-rank): the nprobe nearest
   of all centroids -- the same probe on every rank -- and the estimates of the
   probed lists this rank owns; its top-k' (id, estimate) per query;
2. exchange: all_gather of the ranks' [nq, k'] candidate lists (12 bytes per
   entry: id and estimate);
3. merge (every rank, erq_merge_topk): the global top-k' by (estimate, id) --
   the set the single index keeps, because each owner's top-k' contains all of
   its members of that set;
4. exact re-rank (erq_rerank_ids): each rank computes the exact distances of
   the merged candidates it holds (the others are skipped) and keeps the best
   k; all_gather of the ranks' [nq, k] results;
5. merge (erq_merge_topk): the top-k by (distance, id), the single index's
   answer.

The merges and distances run in the library's kernels; this module only moves
ids between the rank-local and global numbering and calls the collectives.
The arithmetic of a step can be supplied by another backend (``ShardBackend``)
so that the same orchestration runs on CPU ranks in the tests.
"""
from __future__ import annotations

import numpy as np


def partition_lists(sizes, world):
    """Owner rank of every list: greedy by decreasing size (ties by lower list
    id) onto the rank with the fewest rows so far (ties by lower rank)."""
    sizes = np.asarray(sizes, np.int64)
    order = np.lexsort((np.arange(len(sizes)), -sizes))
    load = np.zeros(world, np.int64)
    owner = np.empty(len(sizes), np.int32)
    for c in order:
        r = int(np.argmin(load))
        owner[c] = r
        load[r] += sizes[c]
    return owner


def shard_rows(assign, owner, rank):
    """Global ids (ascending) of the rows whose list this rank owns."""
    return np.nonzero(owner[np.asarray(assign)] == rank)[0].astype(np.int64)


class ShardBackend:
    """Arithmetic of one rank: ``search`` (local ids and estimates of the
    top-k'), ``merge`` (top-k of given (id, value) lists), ``rerank`` (exact
    top-k of given local ids).  Arrays are torch tensors on ``device``."""

    device = "cpu"

    def search(self, Q, kp):
        raise NotImplementedError

    def merge(self, ids, vals, k):
        raise NotImplementedError

    def rerank(self, Q, local_ids, k):
        raise NotImplementedError


class ErqShard(ShardBackend):
    """The library on this rank's GPU: an index over the rank's lists built
    with the global centroids."""

    def __init__(self, index, search_kw, metric="l2"):
        from . import erq
        self.erq = erq
        self.ix = index
        self.kw = dict(search_kw)
        self.metric = metric
        self.device = "cuda"

    def search(self, Q, kp):
        _, _, cids, cest = self.ix.search(Q, kp, rerank_k=0, return_candidates=True, metric=self.metric, **self.kw)
        return cids, cest

    def merge(self, ids, vals, k):
        return self.erq.merge_topk(ids, vals, k, metric=self.metric)

    def rerank(self, Q, local_ids, k):
        return self.ix.rerank_ids(Q, local_ids, k, metric=self.metric)


def _to_global(local, gids):
    """Local row ids -> global ids (-1 stays -1)."""
    import torch
    ok = local >= 0
    out = torch.full_like(local, -1)
    out[ok] = gids[local[ok]]
    return out


def _to_local(glob, g2l):
    """Global ids -> this rank's local ids (-1 where the rank does not hold the row)."""
    import torch
    ok = glob >= 0
    out = torch.full_like(glob, -1)
    out[ok] = g2l[glob[ok]]
    return out


class _DistComm:
    """The exchange over a torch.distributed group (NCCL across GPUs, gloo on CPU)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group

    def world_size(self):
        return self.dist.get_world_size(self.group)

    def all_gather(self, out, t):
        self.dist.all_gather(out, t, group=self.group)


def sharded_search(backend, Q, k, kp, gids, n_total, group=None, comm=None):
    """Steps 1-5 above on this rank; every rank returns the same (ids, values)
    [nq, k] with global ids.  ``gids``: global id of each local row (torch,
    on the backend's device); ``n_total``: rows of the whole index.
    ``comm``: the exchange (world_size(), all_gather(list, tensor)); by
    default torch.distributed on ``group``."""
    import torch
    comm = comm or _DistComm(group)
    world = comm.world_size()
    dev = gids.device
    g2l = torch.full((n_total,), -1, dtype=torch.int64, device=dev)
    g2l[gids] = torch.arange(len(gids), dtype=torch.int64, device=dev)
    lid, lest = backend.search(Q, kp)                              # 1. local top-k'
    cid = _to_global(lid.to(torch.int64), gids)
    all_i = [torch.empty_like(cid) for _ in range(world)]          # 2. exchange
    all_v = [torch.empty_like(lest) for _ in range(world)]
    comm.all_gather(all_i, cid.contiguous())
    comm.all_gather(all_v, lest.contiguous())
    mid, _ = backend.merge(torch.cat(all_i, 1), torch.cat(all_v, 1), kp)   # 3. global top-k'
    rid, rd = backend.rerank(Q, _to_local(mid, g2l), k)           # 4. exact, rows held here
    rid = _to_global(rid, gids)
    all_i = [torch.empty_like(rid) for _ in range(world)]
    all_v = [torch.empty_like(rd) for _ in range(world)]
    comm.all_gather(all_i, rid.contiguous())
    comm.all_gather(all_v, rd.contiguous())
    return backend.merge(torch.cat(all_i, 1), torch.cat(all_v, 1), k)   # 5. the answer
