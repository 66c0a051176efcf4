"""Inner-product metric on the GPU against the FP64 oracle (reading R9 of the
oracle: <o_r, q_r> = <c, q_r> + ||o_r - c|| <o, q_r>, the second factor
estimated as for the distance).

Inner products can be close to zero, so tolerances are absolute per query,
scaled by ||q_r|| * max ||o_r|| (the magnitude of the terms that are summed).
Ids are compared bit-exactly outside near-ties of the measured error."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import check_final_vs_own_candidates, compare_topk_ids, erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _pair(erq, N, D, B, nlist, seed):
    X, lab = S.mixture(N, D, 16, seed, scale="aniso")
    assign = S.kmeans_assign(X, nlist, 4, seed + 7)
    P = S.random_orthogonal(D, seed + 1)
    gx = erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(assign))
    ox = oracle.build_index(X, P, assign, nlist, B)
    return X, gx, ox


def _scale(X, Q):
    return np.linalg.norm(Q.astype(np.float64), axis=1)[:, None] * np.linalg.norm(X.astype(np.float64), axis=1).max()


def _bound16(ox, Q, ids):
    """FP16 rounding of q' = P^T q_r: |f_res|/4 * 2^-11 * sum_i |2 ybar_i| |q'_i|."""
    B = ox["B"]
    qp = Q.astype(np.float64) @ ox["P"].astype(np.float64)
    _, f_res = oracle.stored_factors(ox["stats"])
    rows = ox["row_of"][np.maximum(ids, 0)]
    y2 = 2.0 * ox["codes"][rows].astype(np.float64) - (2 ** B - 1)
    return 0.25 * np.abs(f_res[rows]).astype(np.float64) * np.einsum("qkd,qd->qk", np.abs(y2), np.abs(qp)) * 2.0 ** -11


def _check(gx, ox, X, Q, k, kp, precision, nprobe=None, probe=None, simt=False):
    kw = dict(rerank_k=kp, precision=precision, return_candidates=True, metric="ip", simt_gemm=simt)
    if probe is not None:
        kw["probe"], kw["nprobe"] = to_dev(probe), probe.shape[1]
    else:
        kw["nprobe"] = nprobe
    ids, vals, cids, cest = gx.search(to_dev(Q), k, **kw)
    torch.cuda.synchronize()
    gid, ge = cids.cpu().numpy(), cest.cpu().numpy().astype(np.float64)
    assert (gid >= 0).all()
    assert (np.diff(ge, axis=1) <= 0).all(), "candidates must come in decreasing estimated inner product"
    oest = oracle.estimate_rows(ox, Q, gid, metric="ip")
    sc = _scale(X, Q)
    tol = RTOL * sc
    if precision == "fp16":
        tol = tol + _bound16(ox, Q, gid)
    err = np.abs(ge - oest)
    assert (err <= tol).all(), f"estimates: {np.sum(err > tol)} outside the tolerance (max {np.max(err / sc):.2e})"
    kc = max(k, kp)
    ref = oracle.search(ox, Q, k, kprime=kc + 1, nprobe=nprobe, probe=probe, metric="ip")
    # near-tie radius: the measured error of the query's estimates (FP32), or
    # the FP16 rounding bound of each result
    meas = np.maximum(err.max(axis=1, keepdims=True), 1e-9 * sc)
    rad = np.repeat(meas, kc + 1, axis=1)
    if precision == "fp16":
        rad = rad + _bound16(ox, Q, ref["cand_ids"])
    frac = compare_topk_ids(gid, ref["cand_ids"], ref["cand_est"], what="ip candidates", radius=1.5 * rad,
                            max_excluded=1.0 if precision == "fp16" else 0.05)
    print(f"{precision} ip candidates: {frac:.3f} of slots within the error bound of a neighbour")
    # the selected set is valid: every oracle top-k' id the GPU left out is
    # within the two error bounds of every id it kept instead
    for i in range(len(Q)):
        top = dict(zip(ref["cand_ids"][i, :kc].tolist(), range(kc)))
        mine = dict(zip(gid[i].tolist(), range(kc)))
        missing = [j for o, j in top.items() if o not in mine]
        extra = [j for g, j in mine.items() if g not in top]
        assert len(missing) == len(extra)
        for jo in missing:
            for jg in extra:
                gap = ref["cand_est"][i, jo] - oest[i, jg]          # decreasing order: kept >= left out - bounds
                assert gap <= rad[i, jo] + tol[i, jg] + 1e-9, (i, jo, jg, gap)
    if kp > 0:
        refr = oracle.search(ox, Q, k, kprime=kc, nprobe=nprobe, probe=probe, metric="ip")
        same = (np.sort(gid, 1) == np.sort(ref["cand_ids"][:, :kc], 1)).all(1)
        assert same.mean() > 0.5
        gv = vals.cpu().numpy().astype(np.float64)
        assert (np.diff(gv, axis=1) <= 0).all()
        verr = np.abs(gv[same] - refr["dists"][same])
        assert (verr <= RTOL * sc[same]).all(), "re-ranked inner products"
        compare_topk_ids(ids.cpu().numpy()[same], refr["ids"][same], refr["dists"][same], what="re-ranked ip ids",
                         radius=1.5 * RTOL * np.repeat(sc[same], k, axis=1), max_excluded=0.05)
        # every query's final top-k: the exact re-rank of its own candidates
        check_final_vs_own_candidates(X, Q, gid, ids.cpu().numpy(), gv, k, metric="ip")
    return ids, vals


@pytest.mark.parametrize("precision,B", [("fp32", 5), ("fp16", 5), ("fp16", 3), ("fp32", 7)])
def test_ip_explicit_probe(erq, precision, B):
    X, gx, ox = _pair(erq, 20000, 128, B, 64, 4000 + B)
    Q, _ = S.mixture(300, 128, 16, 4100 + B, comp_seed=4000 + B, scale="aniso")
    probe = S.random_probe_lists(300, 64, 8, 4200 + B)
    _check(gx, ox, X, Q, 10, 32, precision, probe=probe)


@pytest.mark.parametrize("precision,simt", [("fp32", False), ("fp16", False), ("fp32", True)])
def test_ip_probe_by_largest_inner_product(erq, precision, simt):
    """The probe (tensor-core GEMM with a -<q, c> epilogue, or the CUDA-core
    SGEMM) picks the clusters the oracle picks; queries whose nprobe-th and
    (nprobe+1)-th centroid inner products are closer than 1e-4 relative are
    left out (their probe set is decided by rounding)."""
    X, gx, ox = _pair(erq, 30000, 128, 4, 128, 4300)
    Q, _ = S.mixture(400, 128, 16, 4301, comp_seed=4300, scale="aniso")
    nprobe = 6
    cip = Q.astype(np.float64) @ ox["C"].astype(np.float64).T
    srt = -np.sort(-cip, axis=1)
    clean = (srt[:, nprobe - 1] - srt[:, nprobe]) > 1e-4 * np.abs(srt[:, nprobe - 1])
    assert clean.mean() > 0.9
    _check(gx, ox, X, Q[clean], 10, 20, precision, nprobe=nprobe, simt=simt)


def test_ip_full_probe_rerank_is_exact_mips(erq):
    """Probing every cluster and re-ranking 256 candidates returns the exact
    top-10 by inner product (numpy brute force), outside near-ties."""
    X, gx, ox = _pair(erq, 6000, 64, 5, 16, 4400)
    Q, _ = S.mixture(64, 64, 16, 4401, comp_seed=4400, scale="aniso")
    ids, vals = gx.search(to_dev(Q), 10, rerank_k=256, nprobe=16, precision="fp32", metric="ip")
    ip = Q.astype(np.float64) @ X.astype(np.float64).T
    ref = np.stack([np.lexsort((np.arange(len(X)), -row))[:11] for row in ip])
    refv = np.take_along_axis(ip, ref, 1)
    sc = _scale(X, Q)
    assert (np.abs(vals.cpu().numpy() - refv[:, :10]) <= RTOL * sc).all()
    compare_topk_ids(ids.cpu().numpy(), ref, refv, what="exact MIPS", radius=1.5 * RTOL * np.repeat(sc, 11, 1))


@pytest.mark.parametrize("B", [4, 6])
def test_ip_fp8_recall_close_to_fp32(erq, B):
    """The e4m3 scan (B = 4 direct, B = 6 split) ranks by the same
    inner-product estimate."""
    X, gx, ox = _pair(erq, 20000, 128, B, 32, 4500)
    Q, _ = S.mixture(300, 128, 16, 4501, comp_seed=4500, scale="aniso")
    a, _ = gx.search(to_dev(Q), 10, rerank_k=32, nprobe=6, precision="fp32", metric="ip")
    b, _ = gx.search(to_dev(Q), 10, rerank_k=32, nprobe=6, precision="fp8", metric="ip")
    assert (a == b).float().mean().item() > 0.95


def test_ip_rejects_unknown_metric(erq):
    X, gx, ox = _pair(erq, 3000, 64, 4, 8, 4600)
    Q = to_dev(S.mixture(4, 64, 16, 4601, comp_seed=4600, scale="aniso")[0])
    sp = erq.SearchParams()
    sp.k, sp.nprobe, sp.metric = 5, 2, 7
    ids = torch.empty((4, 5), dtype=torch.int64, device=Q.device)
    d = torch.empty((4, 5), dtype=torch.float32, device=Q.device)
    import ctypes as ct
    rc = erq.lib().erq_search(gx._h, ct.c_void_p(Q.data_ptr()), 4, ct.byref(sp), ct.c_void_p(ids.data_ptr()),
                              ct.c_void_p(d.data_ptr()), None)
    assert rc == erq.ERQ_EINVAL


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_cosine_is_the_inner_product_of_unit_vectors(erq, precision):
    """Cosine similarity (Section 7: the method adapts to cosine as RaBitQ
    does): an index built with normalize = 1 holds unit rows (FP64 norm, one
    rounding), the query is scaled to unit length and the inner-product search
    runs; the answer equals the oracle's inner-product search over the same
    unit rows and unit queries, and the values are the exact cosines."""
    X, lab = S.mixture(20000, 128, 16, 4700, scale="aniso")
    assign = S.kmeans_assign(X, 32, 4, 4707)
    P = S.random_orthogonal(128, 4701)
    gx = erq.build_index(to_dev(X), to_dev(P), 5, 32, assign=to_dev(assign), normalize=True)
    Xn = gx.export("raw").numpy()
    X64 = X.astype(np.float64)
    ref_n = (X64 / np.linalg.norm(X64, axis=1, keepdims=True)).astype(np.float32)
    assert np.abs(Xn.astype(np.float64) - ref_n).max() <= 6e-8      # one rounding of the FP64 quotient
    Q, _ = S.mixture(200, 128, 16, 4702, comp_seed=4700, scale="aniso")
    Q = Q * np.float32(3.5)                                          # any query scale
    probe = S.random_probe_lists(200, 32, 6, 4703)
    ids, vals = gx.search(to_dev(Q), 10, rerank_k=40, probe=to_dev(probe), nprobe=6, precision=precision,
                          metric="cos")
    torch.cuda.synchronize()
    Qn = Q.astype(np.float64) / np.linalg.norm(Q.astype(np.float64), axis=1, keepdims=True)
    exact = Qn @ Xn.astype(np.float64).T                             # cosines of the unit rows
    got_i, got_v = ids.cpu().numpy(), vals.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got_v, np.take_along_axis(exact, got_i, 1), atol=2e-6)
    ox = oracle.build_index(Xn, P, assign, 32, 5)
    ref = oracle.search(ox, Qn, 10, kprime=40, probe=probe, metric="ip")
    agree = (got_i == ref["ids"]).mean()
    assert agree >= 0.97, agree                     # differences only where estimates tie at the k'-th candidate
    same = (got_i == ref["ids"]).all(1)
    np.testing.assert_allclose(got_v[same], ref["dists"][same], atol=2e-6)
    gx2 = erq.build_index(to_dev(X[:3000]), to_dev(P), 5, 4, assign=to_dev(assign[:3000] % 4))
    with pytest.raises(erq.ErqError, match="normalize"):
        gx2.search(to_dev(Q[:4]), 10, rerank_k=20, nprobe=2, metric="cos")
