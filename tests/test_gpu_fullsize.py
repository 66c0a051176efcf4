"""Parity at the full size of the 1M x 960 IVF workload (4,096 lists, B = 5,
10,000 queries, nprobe 16, k = 10, exact re-rank of the top 20) in the
configuration the benchmark times (FP16 tensor-core scan, autotuned work
items, asynchronous searches):

* every one of the 10,000 queries: the final top-10 is the exact FP64 re-rank
  of the candidate set the GPU selected (ids and distances);
* 256 seeded queries: every candidate estimate lies within the FP16 bound of
  the FP64 oracle's estimate (oracle codes of the candidate rows, encoded with
  the full set of centroids);
* 24 seeded queries: the candidate sets against the oracle's own top-k' over
  the clusters those queries probe (plus two more each, with the full set of
  centroids), so its answer for them is the full index's."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import check_final_vs_own_candidates, compare_topk_ids, erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _fp16_bound(ox, Q, ids):
    """Per-result bound of the FP16 rounding of q' = P^T q_r (FP64)."""
    B = ox["B"]
    qp = Q.astype(np.float64) @ ox["P"].astype(np.float64)
    _, f_res = oracle.stored_factors(ox["stats"])
    rows = ox["row_of"][np.maximum(ids, 0)]
    y2 = 2.0 * ox["codes"][rows].astype(np.float64) - (2 ** B - 1)
    return 0.5 * np.abs(f_res[rows]).astype(np.float64) * np.einsum("qkd,qd->qk", np.abs(y2), np.abs(qp)) * 2.0 ** -11


def test_fullsize_bench_configuration_sampled(erq):
    cfg = S.WORKLOADS["ivf_n1m_d960_nlist4096"]
    sc = cfg.get("scale", "unit")
    X, _ = S.mixture(cfg["n"], cfg["d"], cfg["n_comp"], cfg["data_seed"], scale=sc)
    Q, _ = S.mixture(cfg["nq"], cfg["d"], cfg["n_comp"], cfg["query_seed"], comp_seed=cfg["data_seed"], scale=sc)
    P = S.random_orthogonal(cfg["d"], cfg["p_seed"])
    dev = torch.device("cuda", 0)
    assign = S.kmeans_assign_torch(X, cfg["nlist"], cfg["kmeans_iters"], 17, sample=cfg["kmeans_sample"], device=dev)
    gx = erq.build_index(to_dev(X), to_dev(P), cfg["B"], cfg["nlist"], assign=to_dev(assign))
    Qd = to_dev(Q)
    k, kp, nprobe = cfg["k"], 20, cfg["nprobes"][0]
    gx.autotune(Qd, k, rerank_k=kp, nprobe=nprobe, precision="fp16")
    for _ in range(3):
        gx.search(Qd, k, rerank_k=kp, nprobe=nprobe, precision="fp16", async_mode=True)
    ids, dists, cids, cest = gx.search(Qd, k, rerank_k=kp, nprobe=nprobe, precision="fp16", async_mode=True,
                                       return_candidates=True)
    torch.cuda.synchronize()
    gx.status()                                  # no device-side error in the asynchronous searches

    C = oracle.centroids(X, assign, cfg["nlist"])
    gid_all = cids.cpu().numpy()
    assert (gid_all >= 0).all()
    # every query: final top-k = exact re-rank of its own candidates
    frac = check_final_vs_own_candidates(X, Q, gid_all, ids.cpu().numpy(), dists.cpu().numpy(), k,
                                         what="full-size re-ranked")
    print(f"full size, all {len(Q)} queries: {frac:.5f} of final slots within a near-tie")
    # 256 queries: estimates of the GPU's candidates against the oracle's
    s256 = np.sort(S.rng(5151).choice(len(Q), 256, replace=False))
    crow = np.unique(gid_all[s256])
    oxc = oracle.build_index(X[crow], P, assign[crow], cfg["nlist"], cfg["B"], centroids_in=C)
    pc = np.searchsorted(crow, gid_all[s256])
    Q256 = Q[s256].astype(np.float64)
    oest = oracle.estimate_rows(oxc, Q256, pc)
    ge = cest.cpu().numpy()[s256].astype(np.float64)
    bound = _fp16_bound(oxc, Q256, pc) + 2e-5 * (np.abs(oest) + 1e-3 * np.median(np.abs(oest)))
    assert (np.abs(ge - oest) <= bound).all(), "estimates outside the FP16 bound"
    probed = np.argsort(oracle.centroid_dists(C, Q256), axis=1, kind="stable")[:, :nprobe + 2]
    for i in range(len(s256)):          # every candidate lies in one of the query's nearest clusters
        assert np.isin(assign[gid_all[s256[i]]], probed[i]).all()
    # 24 queries: candidate sets against the oracle's own top-k'
    cand = np.sort(S.rng(5150).choice(len(Q), 32, replace=False))
    cd = oracle.centroid_dists(C, Q[cand].astype(np.float64))
    srt = np.sort(cd, axis=1)
    # queries whose probe set is not decided by rounding (nprobe-th and next
    # centroid distances more than 1e-5 apart, relative)
    clean = (srt[:, nprobe] - srt[:, nprobe - 1]) > 1e-5 * srt[:, nprobe]
    assert clean.mean() > 0.8
    sample = cand[clean][:24]
    Qs = Q[sample].astype(np.float64)
    order = np.argsort(oracle.centroid_dists(C, Qs), axis=1, kind="stable")
    probe = order[:, :nprobe]
    rows = np.nonzero(np.isin(assign, np.unique(order[:, :nprobe + 2])))[0]   # sorted global ids
    ox = oracle.build_index(X[rows], P, assign[rows], cfg["nlist"], cfg["B"], centroids_in=C)

    gid = cids.cpu().numpy()[sample]
    assert (gid >= 0).all()
    pos = np.searchsorted(rows, gid)
    assert (pos < len(rows)).all() and (rows[np.minimum(pos, len(rows) - 1)] == gid).all(), \
        "every GPU candidate lies in a cluster the oracle probes"
    oest = oracle.estimate_rows(ox, Qs, pos)
    ge = cest.cpu().numpy()[sample].astype(np.float64)
    bound = _fp16_bound(ox, Qs, pos) + 2e-5 * (np.abs(oest) + 1e-3 * np.median(np.abs(oest)))
    assert (np.abs(ge - oest) <= bound).all(), "estimates outside the FP16 bound"

    ref = oracle.search(ox, Qs, k, kprime=kp + 1, nprobe=nprobe)
    np.testing.assert_array_equal(ref["probe"][:, :nprobe], probe)
    rad = _fp16_bound(ox, Qs, ref["cand_ids"]) + 2e-5 * np.abs(ref["cand_est"])
    compare_topk_ids(pos, ref["cand_ids"], ref["cand_est"], what="full-size candidates", radius=rad,
                     max_excluded=1.0)
    refr = oracle.search(ox, Qs, k, kprime=kp, nprobe=nprobe)
    same = (np.sort(pos, 1) == np.sort(ref["cand_ids"][:, :kp], 1)).all(1)
    assert same.mean() > 0.5
    gi = np.searchsorted(rows, ids.cpu().numpy()[sample])
    gd = dists.cpu().numpy()[sample].astype(np.float64)
    derr = np.abs(gd[same] - refr["dists"][same]) / np.abs(refr["dists"][same])
    assert derr.max(initial=0.0) <= 1e-5
    compare_topk_ids(gi[same], refr["ids"][same], refr["dists"][same], 1.5 * max(derr.max(initial=0.0), 1e-7),
                     "full-size re-ranked ids", max_excluded=0.05)
