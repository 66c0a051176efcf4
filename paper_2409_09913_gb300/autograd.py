"""Differentiable estimated scores (query tower training against a compressed corpus).

``EstimatedScores.apply(Q, index, ids)`` returns est(q_i, ids[i, j]) (Eq. 3.3 with
Eq. eq:dis to ip, FP32 path) and back-propagates to Q through
erq_search_backward: d est / d q_r = 2 (q_r - c) + f_res P ybar, with codes and
ids fixed.  Only Q and ids are saved: the backward recomputes everything else
from the index ("recompute in backward"), so the saved state is
nq * (D * 4 + k * 8) bytes instead of the k codes per query.
"""
from __future__ import annotations

import torch

from .erq import Index


class EstimatedScores(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q: torch.Tensor, index: Index, ids: torch.Tensor):
        Qc = Q.detach().contiguous()
        est = index.estimate(Qc, ids)
        ctx.index = index
        ctx.save_for_backward(Qc, ids)
        return est

    @staticmethod
    def backward(ctx, grad):
        Q, ids = ctx.saved_tensors
        gQ = ctx.index.search_backward(Q, ids, grad.contiguous().float())
        return gQ, None, None


def search_scores(index: Index, Q: torch.Tensor, k: int, **search_kw):
    """Search (no gradient through the discrete selection), then differentiable
    estimated scores of the returned candidates.  Returns (ids, scores)."""
    with torch.no_grad():
        _, _, cand_ids, _ = index.search(Q.detach(), k, return_candidates=True, **search_kw)
    ids = cand_ids[:, :k].contiguous()
    return ids, EstimatedScores.apply(Q, index, ids)
