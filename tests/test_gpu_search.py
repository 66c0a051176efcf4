"""GPU parity of the search path against the FP64 oracle.

Estimated candidates (ids + estimates) and re-ranked results are compared on
the same seeded inputs: ids bit-exactly wherever the oracle's ranking is not
decided by a near-tie, estimates and distances within the FP32 tolerance."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import FP32_RTOL, assert_close_rel, check_final_vs_own_candidates, compare_topk_ids, erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _build_pair(erq, N, D, B, nlist, seed, n_comp=None, scale="unit"):
    X, lab = S.mixture(N, D, n_comp or max(2, nlist), seed, scale=scale)
    assign = S.kmeans_assign(X, nlist, 4, seed + 7) if nlist > 1 else np.zeros(N, np.int32)
    P = S.random_orthogonal(D, seed + 1)
    gx = erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(assign))
    ox = oracle.build_index(X, P, assign, nlist, B)
    return X, P, assign, gx, ox


def _check_search(erq, gx, ox, Q, k, kp, nprobe=None, probe=None, precision="fp32", rtol=FP32_RTOL):
    kw = dict(rerank_k=kp, precision=precision, return_candidates=True)
    if probe is not None:
        kw["probe"] = to_dev(probe)
        kw["nprobe"] = probe.shape[1]
    else:
        kw["nprobe"] = nprobe
    ids, dists, cids, cest = gx.search(to_dev(Q), k, **kw)
    torch.cuda.synchronize()
    kc = max(k, kp)
    ref = oracle.search(ox, Q, k, kprime=kc + 1, nprobe=nprobe, probe=probe)
    # estimates of the ids the GPU returned, recomputed by the oracle (FP64)
    ce = cest.cpu().numpy()
    gid = cids.cpu().numpy()
    oest = oracle.estimate_rows(ox, Q, np.where(gid >= 0, gid, -1))
    ok = gid >= 0
    err = assert_close_rel(ce[ok], oest[ok], rtol, "estimates")
    # ids: bit-exact except where the oracle's values are closer than twice the
    # measured error (one extra oracle column exposes ties across the cut)
    radius = 1.5 * max(err, 1e-7)
    compare_topk_ids(gid, ref["cand_ids"], ref["cand_est"], radius, "estimated candidates", max_excluded=0.05)
    if kp > 0:
        refr = oracle.search(ox, Q, k, kprime=kc, nprobe=nprobe, probe=probe)
        gd = dists.cpu().numpy()
        # re-ranked ids: same candidate sets -> exact distances decide
        same = (np.sort(cids.cpu().numpy(), 1) == np.sort(ref["cand_ids"][:, :kc], 1)).all(1)
        gi = ids.cpu().numpy()
        assert same.mean() > 0.9
        derr = assert_close_rel(gd[same], refr["dists"][same], rtol, "re-ranked distances")
        compare_topk_ids(gi[same], refr["ids"][same], refr["dists"][same], 1.5 * max(derr, 1e-7), "re-ranked ids",
                         max_excluded=0.05)
        # every query's final top-k: the exact re-rank of its own candidate set
        check_final_vs_own_candidates(ox["X"], Q, gid, gi, gd, k)
    return ids, dists, cids, cest


def test_bruteforce_config_small(erq):
    """No IVF (one cluster, c = mean): N=10,000, D=128, B=4, 100 queries,
    top-10 after exact re-rank of the estimated top-100."""
    cfg = S.WORKLOADS["bruteforce_n10k_d128_b4"]
    X, lab = S.mixture(cfg["n"], cfg["d"], cfg["n_comp"], cfg["data_seed"])
    Q, _ = S.mixture(cfg["nq"], cfg["d"], cfg["n_comp"], cfg["query_seed"], comp_seed=cfg["data_seed"])
    P = S.random_orthogonal(cfg["d"], cfg["p_seed"])
    assign = np.zeros(cfg["n"], np.int32)
    gx = erq.build_index(to_dev(X), to_dev(P), cfg["B"], 1, assign=to_dev(assign))
    ox = oracle.build_index(X, P, assign, 1, cfg["B"])
    ids, dists, _, _ = _check_search(erq, gx, ox, Q, cfg["k"], cfg["rerank_k"], nprobe=1)
    gt, _ = oracle.exact_knn(X, Q, cfg["k"])
    recall = np.mean([len(set(a) & set(b)) / cfg["k"] for a, b in zip(ids.cpu().numpy(), gt)])
    assert recall > 0.98


@pytest.mark.parametrize("B", [3, 5, 7, 9])
def test_ivf_explicit_probe(erq, B):
    """IVF with probe lists drawn by the generator (both sides scan the same clusters)."""
    X, P, assign, gx, ox = _build_pair(erq, 20000, 128, B, 64, 500 + B, n_comp=16, scale="aniso")
    Q, _ = S.mixture(150, 128, 16, 600 + B, comp_seed=500 + B, scale="aniso")
    probe = S.random_probe_lists(150, 64, 8, 700 + B)
    _check_search(erq, gx, ox, Q, 10, 40, probe=probe)


def test_ivf_computed_probe(erq):
    """The GPU's own centroid search: probe sets equal the oracle's except where
    the oracle's centroid distances are within FP32 noise at the cut."""
    X, P, assign, gx, ox = _build_pair(erq, 20000, 192, 4, 50, 800, n_comp=12, scale="aniso")
    Q, _ = S.mixture(200, 192, 12, 801, comp_seed=800, scale="aniso")
    nprobe = 6
    ids, dists, cids, cest = gx.search(to_dev(Q), 10, rerank_k=30, nprobe=nprobe, return_candidates=True)
    cd = oracle.centroid_dists(ox["C"], Q)
    srt = np.sort(cd, 1)
    clean = (srt[:, nprobe] - srt[:, nprobe - 1]) > 1e-4 * srt[:, nprobe]
    assert clean.mean() > 0.9
    ref = oracle.search(ox, Q[clean], 10, kprime=31, nprobe=nprobe)
    gid = cids.cpu().numpy()[clean]
    oest = oracle.estimate_rows(ox, Q[clean], gid)
    err = assert_close_rel(cest.cpu().numpy()[clean], oest, FP32_RTOL, "estimates")
    compare_topk_ids(gid, ref["cand_ids"], ref["cand_est"], 1.5 * max(err, 1e-7), "candidates", max_excluded=0.05)


@pytest.mark.parametrize("nprobe", [40, 150])
def test_ivf_computed_probe_wide(erq, nprobe):
    """Probe lists longer than a warp (the block-per-query radix selection over
    400 centroid distances): as above, probe sets equal the oracle's outside
    FP32 noise at the cut."""
    X, P, assign, gx, ox = _build_pair(erq, 20000, 128, 4, 400, 820, n_comp=40, scale="aniso")
    Q, _ = S.mixture(150, 128, 40, 821, comp_seed=820, scale="aniso")
    ids, dists, cids, cest = gx.search(to_dev(Q), 10, rerank_k=30, nprobe=nprobe, return_candidates=True)
    cd = oracle.centroid_dists(ox["C"], Q)
    srt = np.sort(cd, 1)
    clean = (srt[:, nprobe] - srt[:, nprobe - 1]) > 1e-4 * srt[:, nprobe]
    assert clean.sum() >= 100              # (the cut falls in a denser part of the distances at 150)
    ref = oracle.search(ox, Q[clean], 10, kprime=31, nprobe=nprobe)
    gid = cids.cpu().numpy()[clean]
    oest = oracle.estimate_rows(ox, Q[clean], gid)
    err = assert_close_rel(cest.cpu().numpy()[clean], oest, FP32_RTOL, "estimates")
    compare_topk_ids(gid, ref["cand_ids"], ref["cand_est"], 1.5 * max(err, 1e-7), "candidates", max_excluded=0.05)


def test_variable_nprobe_and_large_k(erq):
    """Per-query nprobe, k' larger than some probed clusters, -1 padding."""
    X, P, assign, gx, ox = _build_pair(erq, 3000, 64, 5, 40, 900)
    Q, _ = S.mixture(30, 64, 40, 901, comp_seed=900)
    probe = S.random_probe_lists(30, 40, 6, 902)
    npq = S.uniform_ints(30, 1, 6, 903)
    k, kp = 20, 150
    ids, dists, cids, cest = gx.search(to_dev(Q), k, rerank_k=kp, probe=to_dev(probe), nprobe=6,
                                       nprobe_per_query=to_dev(npq), return_candidates=True)
    gid = cids.cpu().numpy()
    oest = oracle.estimate_rows(ox, Q, np.where(gid >= 0, gid, -1))
    err = assert_close_rel(cest.cpu().numpy()[gid >= 0], oest[gid >= 0], FP32_RTOL, "estimates")
    for i in range(30):
        ref = oracle.search(ox, Q[i:i + 1], k, kprime=kp + 1, probe=probe[i:i + 1, :npq[i]])
        compare_topk_ids(gid[i:i + 1], ref["cand_ids"], ref["cand_est"], 1.5 * max(err, 1e-7), "cands",
                         max_excluded=0.05)
        n_avail = sum(np.diff(ox["list_off"])[c] for c in probe[i, :npq[i]])
        assert (cids[i].cpu().numpy() >= 0).sum() == min(kp, n_avail)


def test_no_rerank_returns_estimates(erq):
    X, P, assign, gx, ox = _build_pair(erq, 4000, 64, 6, 8, 1000)
    Q, _ = S.mixture(20, 64, 8, 1001, comp_seed=1000)
    ids, dists = gx.search(to_dev(Q), 10, rerank_k=0, nprobe=3)
    ref = oracle.search(ox, Q, 10, kprime=11, nprobe=3)
    cd = oracle.centroid_dists(ox["C"], Q)
    srt = np.sort(cd, 1)
    clean = (srt[:, 3] - srt[:, 2]) > 1e-4 * srt[:, 3]
    assert clean.mean() > 0.8
    gid = ids.cpu().numpy()[clean]
    oest = oracle.estimate_rows(ox, Q[clean], gid)
    err = assert_close_rel(dists.cpu().numpy()[clean], oest, FP32_RTOL, "estimated distances")
    compare_topk_ids(gid, ref["cand_ids"][clean], ref["cand_est"][clean], 1.5 * max(err, 1e-7), "ids",
                     max_excluded=0.05)


def test_search_host_matches_device(erq):
    X, P, assign, gx, ox = _build_pair(erq, 3000, 64, 4, 4, 1100)
    Q, _ = S.mixture(16, 64, 4, 1101, comp_seed=1100)
    a_ids, a_d = gx.search(to_dev(Q), 5, rerank_k=20, nprobe=2)
    b_ids, b_d = gx.search_host(torch.from_numpy(Q).pin_memory(), 5, rerank_k=20, nprobe=2)
    assert torch.equal(a_ids.cpu(), b_ids) and torch.equal(a_d.cpu(), b_d)


def test_estimate_pairs(erq):
    X, P, assign, gx, ox = _build_pair(erq, 2000, 128, 5, 5, 1200)
    Q, _ = S.mixture(7, 128, 5, 1201, comp_seed=1200)
    ids = np.stack([S.rng(1202 + i).choice(2000, 33, replace=False) for i in range(7)]).astype(np.int64)
    ids[0, 3] = -1
    est = gx.estimate(to_dev(Q), to_dev(ids)).cpu().numpy()
    ref = oracle.estimate_rows(ox, Q, ids)
    assert np.isnan(est[0, 3])
    m = ids >= 0
    assert_close_rel(est[m], ref[m], FP32_RTOL, "pair estimates")


def test_edge_cases_and_errors(erq):
    X, P, assign, gx, ox = _build_pair(erq, 1000, 64, 4, 4, 1300)
    Q = to_dev(S.mixture(3, 64, 4, 1301, comp_seed=1300)[0])
    ids, d = gx.search(Q[:0], 5, nprobe=2)                      # empty batch
    assert ids.shape == (0, 5)
    ids, d = gx.search(Q, 5, rerank_k=5, nprobe=4)               # nprobe == nlist
    assert (ids >= 0).all()
    for bad in (dict(k=0, nprobe=2), dict(k=5, nprobe=5), dict(k=5, nprobe=0), dict(k=5, rerank_k=3, nprobe=2)):
        k = bad.pop("k")
        with pytest.raises(erq.ErqError):
            gx.search(Q, k, **bad)
    with pytest.raises(erq.ErqError, match="kind::i8"):
        gx.search(Q, 5, nprobe=2, precision="int8")
    bad_probe = torch.tensor([[0, 9], [1, 2], [2, 3]], dtype=torch.int32, device="cuda")
    with pytest.raises(erq.ErqError, match="bound"):
        gx.search(Q, 5, probe=bad_probe, nprobe=2)
    # the index stays usable after a reported device-side error
    ids, d = gx.search(Q, 5, rerank_k=10, nprobe=2)
    assert (ids >= 0).all()
    nr = erq.build_index(to_dev(X), to_dev(P), 4, 4, assign=to_dev(assign), keep_raw=False)
    with pytest.raises(erq.ErqError, match="keep_raw"):
        nr.search(Q, 5, rerank_k=10, nprobe=2)


def test_kmeans_build_runs_and_partitions(erq):
    """assign = NULL: the library trains k-means itself (outside parity); the
    index must be a valid partition and searchable."""
    X, _ = S.mixture(20000, 64, 16, 1400)
    P = S.random_orthogonal(64, 1401)
    gx = erq.build_index(to_dev(X), to_dev(P), 4, 32, kmeans_iters=5, kmeans_sample=8000)
    off = gx.export("list_offsets").numpy()
    ids = gx.export("list_ids").numpy()
    assert off[0] == 0 and off[-1] == 20000 and (np.diff(off) >= 0).all()
    assert np.array_equal(np.sort(ids), np.arange(20000))
    Q = to_dev(S.mixture(50, 64, 16, 1402, comp_seed=1400)[0])
    res, _ = gx.search(Q, 10, rerank_k=50, nprobe=8)
    gt, _ = oracle.exact_knn(X, Q.cpu().numpy(), 10)
    recall = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(res.cpu().numpy(), gt)])
    assert recall > 0.8


def test_tensor_core_gemm_matches_simt(erq):
    """The FP32-accurate tensor-core GEMM (hi/lo FP16 split) used for the query
    rotation and centroid distances agrees with the CUDA-core SGEMM to FP32
    precision, so estimates and probe lists agree."""
    X, P, assign, gx, ox = _build_pair(erq, 8000, 256, 5, 32, 1500, scale="aniso")
    Q, _ = S.mixture(300, 256, 32, 1501, comp_seed=1500, scale="aniso")
    a = gx.search(to_dev(Q), 10, rerank_k=30, nprobe=5, return_candidates=True)
    b = gx.search(to_dev(Q), 10, rerank_k=30, nprobe=5, return_candidates=True, simt_gemm=True)
    ok = (a[2] == b[2]).all(1).cpu().numpy()
    assert ok.mean() > 0.95
    assert_close_rel(a[3].cpu().numpy()[ok], b[3].cpu().numpy()[ok], FP32_RTOL, "tc vs simt estimates")
    oest = oracle.estimate_rows(ox, Q, a[2].cpu().numpy())
    assert_close_rel(a[3].cpu().numpy(), oest, FP32_RTOL, "tc-gemm estimates vs oracle")


def test_probe_ties_take_lower_cluster(erq):
    """Identical centroids (a cluster duplicated) tie exactly; the probe keeps
    the lower cluster id, as the oracle does."""
    X, lab = S.mixture(2000, 64, 6, 1600)
    assign = S.kmeans_assign(X, 6, 4, 1601)
    X2 = np.concatenate([X, X])
    a2 = np.concatenate([assign, assign + 6]).astype(np.int32)
    P = S.random_orthogonal(64, 1602)
    gx = erq.build_index(to_dev(X2), to_dev(P), 4, 12, assign=to_dev(a2))
    ox = oracle.build_index(X2, P, a2, 12, 4)
    Q, _ = S.mixture(40, 64, 6, 1603, comp_seed=1600)
    members = [set(np.nonzero(a2 == c)[0].tolist()) for c in range(12)]
    for nprobe in (1, 3, 5):
        ids, _, cids, cest = gx.search(to_dev(Q), 5, rerank_k=0, nprobe=nprobe, return_candidates=True)
        ref = oracle.search(ox, Q, 5, kprime=6, nprobe=nprobe)
        got = cids.cpu().numpy()
        for i in range(len(Q)):
            # with an odd nprobe the last probe slot falls inside a tied pair: the
            # GPU must have taken the lower cluster id, exactly as the oracle did
            allowed = set().union(*(members[c] for c in ref["probe"][i, :nprobe]))
            assert set(got[i].tolist()) <= allowed, (nprobe, i, ref["probe"][i, :nprobe])


def test_probe_far_orthogonal_queries(erq):
    """Queries far from every centroid and orthogonal to all of them, so all
    centroid distances agree to ~1e-8 relative: the probed clusters must be
    among the oracle's nearest up to FP32 rounding, for nprobe below and
    above the number of 32-cluster groups."""
    D, nl = 64, 64
    rng = np.random.default_rng(1700)
    cent = np.zeros((nl, D), np.float32)
    for j in range(nl):
        cent[j, 1 + j // 2] = 1.0 if j % 2 == 0 else -1.0
    assign = np.repeat(np.arange(nl, dtype=np.int32), 40)
    X = (cent[assign] + 1e-3 * rng.standard_normal((len(assign), D))).astype(np.float32)
    X[:, 0] = 0.0
    P = S.random_orthogonal(D, 1701)
    gx = erq.build_index(to_dev(X), to_dev(P), 4, nl, assign=to_dev(assign))
    ox = oracle.build_index(X, P, assign, nl, 4)
    Q = np.zeros((20, D), np.float32)
    Q[:, 0] = 100.0
    Q[:, 1:] = 1e-4 * rng.standard_normal((20, D - 1))
    cd = oracle.centroid_dists(ox["C"], Q)
    for nprobe in (1, 5, 32):
        ids, _, cids, _ = gx.search(to_dev(Q), 5, rerank_k=0, nprobe=nprobe, return_candidates=True)
        torch.cuda.synchronize()
        kth = np.sort(cd, 1)[:, nprobe - 1]
        got = cids.cpu().numpy()                      # original row ids of the candidates
        for i in range(len(Q)):
            for r in got[i]:
                c = int(assign[r])
                assert cd[i, c] <= kth[i] * (1 + 1e-6), (nprobe, i, c, cd[i, c], kth[i])


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_async_mode_and_cuda_graph(erq, precision):
    """ERQ_SEARCH_ASYNC sizes its buffers from host-side bounds (no read-back),
    returns the same results as the synchronous call, and can be recorded into
    a CUDA graph whose replay searches new queries."""
    X, P, assign, gx, ox = _build_pair(erq, 12000, 128, 5, 48, 1700, scale="aniso")
    Q1, _ = S.mixture(400, 128, 48, 1701, comp_seed=1700, scale="aniso")
    Q2, _ = S.mixture(400, 128, 48, 1702, comp_seed=1700, scale="aniso")
    kw = dict(rerank_k=20, nprobe=6, precision=precision)
    ref1 = gx.search(to_dev(Q1), 10, **kw)
    ref2 = gx.search(to_dev(Q2), 10, **kw)
    a1 = gx.search(to_dev(Q1), 10, async_mode=True, **kw)       # also sizes the buffers
    torch.cuda.synchronize()
    assert torch.equal(a1[0], ref1[0]) and torch.equal(a1[1], ref1[1])
    static_q = to_dev(Q1).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gx.search(static_q, 10, async_mode=True, **kw)          # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out_ids, out_d = gx.search(static_q, 10, async_mode=True, **kw)
    static_q.copy_(to_dev(Q2))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out_ids, ref2[0]) and torch.equal(out_d, ref2[1])
    gx.status()                                                 # no device-side error was recorded
