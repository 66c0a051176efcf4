"""Differentiable estimated scores (query tower training against a compressed corpus).

``EstimatedScores.apply(Q, index, ids)`` returns est(q_i, ids[i, j]) (Eq. 3.3 with
Eq. eq:dis to ip, FP32 path) and back-propagates to Q through
erq_search_backward: d est / d q_r = 2 (q_r - c) + f_res P ybar, with codes and
ids fixed.  ``EstimatedScores.apply(Q, index, ids, "ip")`` does the same for the
estimated inner products <c, q_r> - (f_res / 2) <ybar, P^T q_r>, whose gradient
is c - (f_res / 2) P ybar.  Only Q and ids are saved: the backward recomputes everything else
from the index ("recompute in backward"), so the saved state is
nq * (D * 4 + k * 8) bytes instead of the k codes per query.
"""
from __future__ import annotations

import torch

from .erq import Index


class EstimatedScores(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q: torch.Tensor, index: Index, ids: torch.Tensor, metric: str = "l2"):
        Qc = Q.detach().contiguous()
        est = index.estimate(Qc, ids, metric=metric)
        ctx.index = index
        ctx.metric = metric
        ctx.save_for_backward(Qc, ids)
        return est

    @staticmethod
    def backward(ctx, grad):
        Q, ids = ctx.saved_tensors
        gQ = ctx.index.search_backward(Q, ids, grad.contiguous().float(), metric=ctx.metric)
        return gQ, None, None, None


def search_scores(index: Index, Q: torch.Tensor, k: int, metric: str = "l2", **search_kw):
    """Search (no gradient through the discrete selection), then differentiable
    estimated scores of the returned candidates.  Returns (ids, scores)."""
    with torch.no_grad():
        _, _, cand_ids, _ = index.search(Q.detach(), k, return_candidates=True, metric=metric, **search_kw)
    ids = cand_ids[:, :k].contiguous()
    return ids, EstimatedScores.apply(Q, index, ids, metric)
