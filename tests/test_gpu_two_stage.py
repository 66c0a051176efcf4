"""Two-stage (MSB-first) search (Section 4.2) on the GPU against the oracle's
two_stage_search.

Stage-1 quantities are FP32 on the GPU and FP64 in the oracle, so the pruning
decision est1 - bound > tau and the ranking of the survivors are compared
outside near-ties: every GPU candidate is an oracle survivor up to the FP32
tolerance, every oracle candidate the GPU left out is near the pruning
threshold or near the k'-th estimate, the candidates' estimates are the
oracle's full estimates within 1e-5, and every query's final top-k is the
exact re-rank of its own candidates."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import assert_close_rel, check_final_vs_own_candidates, compare_topk_ids, erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _index(erq, N, D, B, nlist, seed):
    X, _ = S.mixture(N, D, 16, seed, scale="aniso")
    assign = S.kmeans_assign(X, nlist, 4, seed + 7)
    P = S.random_orthogonal(D, seed + 1)
    gx = erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(assign))
    return X, gx, oracle.build_index(X, P, assign, nlist, B)


def _oracle_rows(ox, Q, probe, eps0):
    """Per query: global ids, est1, bound and full estimate of every probed row (FP64)."""
    out = []
    for i in range(len(Q)):
        parts = []
        for c in probe[i]:
            if c < 0:
                continue
            rows = np.arange(ox["list_off"][c], ox["list_off"][c + 1])
            if len(rows):
                r = oracle.two_stage_rows(ox, Q[i], c, rows, eps0)
                parts.append((ox["list_ids"][rows], r["est1"], r["bound"], r["est"]))
        out.append(tuple(np.concatenate(x) for x in zip(*parts)))
    return out


@pytest.mark.parametrize("D,B,kp,eps0", [(128, 5, 40, 1.9), (192, 7, 24, 1.9), (128, 3, 32, 1.0), (64, 8, 100, 2.5),
                                         (128, 1, 20, 1.9), (256, 6, 40, 0.5), (128, 9, 32, 1.9)])
def test_two_stage_matches_oracle(erq, D, B, kp, eps0):
    X, gx, ox = _index(erq, 20000, D, B, 64, 5000 + D + B)
    nq, nprobe, k = 200, 6, 10
    Q, _ = S.mixture(nq, D, 16, 5100 + D, comp_seed=5000 + D + B, scale="aniso")
    ids, dists, cids, cest, (rows, surv) = gx.search_two_stage(to_dev(Q), k, rerank_k=kp, nprobe=nprobe, eps0=eps0,
                                                                return_candidates=True, return_stats=True)
    torch.cuda.synchronize()
    ref = oracle.two_stage_search(ox, Q, k, kp, nprobe=nprobe, eps0=eps0)
    assert rows == int(ref["rows"].sum())
    assert abs(surv - int(ref["survivors"].sum())) <= max(2, 0.002 * surv), (surv, ref["survivors"].sum())
    gid = cids.cpu().numpy()
    ge = cest.cpu().numpy().astype(np.float64)
    have = gid >= 0
    n_exp = np.minimum(ref["survivors"], kp)
    assert (have.sum(1) >= n_exp - 2).all()
    # the candidates' estimates are the full B-bit estimates (Eq. 4.2 = Eq. 3.3)
    oest = oracle.estimate_rows(ox, Q, np.where(have, gid, 0))
    assert_close_rel(ge[have], oest[have], 1e-5, "two-stage candidate estimates")
    per = _oracle_rows(ox, Q, ref["probe"], eps0)
    for i in range(nq):
        gids, e1, bd, est = per[i]
        scale = np.abs(est).max() + 1e-30
        tol = 2e-5 * scale
        lb = e1 - bd
        pos = dict(zip(gids.tolist(), range(len(gids))))
        tau = ref["tau"][i]
        mine = set(gid[i][have[i]].tolist())
        top = set(ref["cand_ids"][i][ref["cand_ids"][i] >= 0].tolist())
        kth = ref["cand_est"][i][np.isfinite(ref["cand_est"][i])].max(initial=-np.inf)
        for g in mine - top:                       # kept by the GPU only: a survivor, near a cut
            j = pos[g]
            assert lb[j] <= tau + tol, (i, g, lb[j], tau)
            assert est[j] <= kth + tol or abs(lb[j] - tau) <= tol, (i, g)
        for o in top - mine:                       # left out by the GPU: near the prune or rank cut
            j = pos[o]
            assert abs(lb[j] - tau) <= tol or est[j] >= kth - tol, (i, o, lb[j], tau, est[j], kth)
    frac = check_final_vs_own_candidates(X, Q, gid, ids.cpu().numpy(), dists.cpu().numpy(), k)
    print(f"two-stage B={B} eps0={eps0}: survivors {surv}/{rows}, final near-tie slots {frac:.4f}")


def test_two_stage_without_pruning_is_the_single_stage_search(erq):
    """eps0 = inf keeps every probed row: the FP32 scan's candidates and answer."""
    X, gx, ox = _index(erq, 15000, 128, 5, 48, 5200)
    Q, _ = S.mixture(150, 128, 16, 5201, comp_seed=5200, scale="aniso")
    a_ids, a_d, a_c, a_e = gx.search(to_dev(Q), 10, rerank_k=30, nprobe=5, precision="fp32", return_candidates=True)
    b_ids, b_d, b_c, b_e, (rows, surv) = gx.search_two_stage(to_dev(Q), 10, rerank_k=30, nprobe=5,
                                                             eps0=float("inf"), return_candidates=True,
                                                             return_stats=True)
    torch.cuda.synchronize()
    assert surv == rows
    assert_close_rel(b_e.cpu().numpy(), a_e.cpu().numpy(), 1e-5, "estimates")
    ref = oracle.search(ox, Q, 10, kprime=30, nprobe=5)
    # near-ties: within 1.5x the largest measured error of the GPU's own estimates
    err = assert_close_rel(b_e.cpu().numpy(), oracle.estimate_rows(ox, Q, b_c.cpu().numpy()), 1e-5, "vs oracle")
    compare_topk_ids(b_c.cpu().numpy(), ref["cand_ids"], ref["cand_est"], 1.5 * max(err, 1e-7), "candidates",
                     max_excluded=0.03)
    compare_topk_ids(b_ids.cpu().numpy(), ref["ids"], ref["dists"], 1e-5, "ids", max_excluded=0.01)


def test_two_stage_edge_cases(erq):
    """One query with one probed list and k' above its rows (tau = +inf: every
    row survives), and the rejected configurations (eps0 < 0, B = 4, the
    inner-product metric)."""
    X, gx, ox = _index(erq, 3000, 64, 5, 40, 5300)
    Q, _ = S.mixture(1, 64, 16, 5301, comp_seed=5300, scale="aniso")
    ids, d, (rows, surv) = gx.search_two_stage(to_dev(Q), 10, rerank_k=1000, nprobe=1, eps0=1.9, return_stats=True)
    torch.cuda.synchronize()
    ref = oracle.two_stage_search(ox, Q, 10, 1000, nprobe=1, eps0=1.9)
    assert rows == int(ref["rows"][0]) and surv == rows           # fewer rows than k': tau = inf
    compare_topk_ids(ids.cpu().numpy(), ref["ids"], ref["dists"], 1e-5, "ids")
    with pytest.raises(erq.ErqError):
        gx.search_two_stage(to_dev(Q), 10, rerank_k=20, nprobe=2, eps0=-1.0)
    X4, gx4, _ = _index(erq, 3000, 64, 4, 8, 5310)
    with pytest.raises(erq.ErqError, match="B = 4"):
        gx4.search_two_stage(to_dev(Q), 10, rerank_k=20, nprobe=2)
    sp = erq.SearchParams()
    sp.k, sp.rerank_k, sp.nprobe, sp.metric = 10, 20, 2, 1
    import ctypes as ct
    Qd = to_dev(Q)
    o_i = torch.empty((1, 10), dtype=torch.int64, device=Qd.device)
    o_d = torch.empty((1, 10), dtype=torch.float32, device=Qd.device)
    rc = erq.lib().erq_search_two_stage(gx._h, ct.c_void_p(Qd.data_ptr()), 1, ct.byref(sp), ct.c_float(1.9),
                                        ct.c_void_p(o_i.data_ptr()), ct.c_void_p(o_d.data_ptr()), None, None)
    assert rc == erq.ERQ_EUNSUPPORTED
