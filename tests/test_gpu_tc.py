"""Tensor-core (tcgen05 kind::f16) scan against the FP64 oracle.

The FP16 path is exact in the codes (2*ybar is an odd integer <= 255) and
rounds only the rotated query q' to FP16, so every estimate must lie within a
per-result bound derived from that rounding:
    |est_gpu - est| <= |f_res|/2 * 2^-11 * sum_i |2 ybar_i| |q'_i|  (+ FP32 slack).
Ids are compared bit-exactly outside near-ties of that size, and the
re-ranked top-k must match the oracle's exact re-rank."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import assert_close_rel, check_final_vs_own_candidates, compare_topk_ids, erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _index(erq, N, D, B, nlist, seed):
    X, lab = S.mixture(N, D, 16, seed, scale="aniso")
    assign = S.kmeans_assign(X, nlist, 4, seed + 7)
    P = S.random_orthogonal(D, seed + 1)
    return X, P, erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(assign)), \
        oracle.build_index(X, P, assign, nlist, B)


def _bound(ox, Q, ids):
    """Per-result bound of the FP16 query rounding (FP64)."""
    B = ox["B"]
    qp = Q.astype(np.float64) @ ox["P"].astype(np.float64)          # q' = P^T q_r (rows)
    _, f_res = oracle.stored_factors(ox["stats"])
    rows = ox["row_of"][np.maximum(ids, 0)]
    y2 = 2.0 * ox["codes"][rows].astype(np.float64) - (2 ** B - 1)   # [nq, k, D]
    s = np.einsum("qkd,qd->qk", np.abs(y2), np.abs(qp))
    return 0.5 * np.abs(f_res[rows]).astype(np.float64) * s * 2.0 ** -11


@pytest.mark.parametrize("D,B,nq,kp", [(128, 5, 1500, 32), (64, 3, 400, 32), (960, 7, 300, 32), (128, 5, 600, 100),
                                       (64, 4, 300, 128)])
def test_tc_scan_within_fp16_bound(erq, D, B, nq, kp):
    """k' <= 32 runs the 64-query / 64-entry-list configuration of the scan,
    larger k' the 32-query / 160-entry-list one."""
    X, P, gx, ox = _index(erq, 20000, D, B, 64, 3000 + D + B)
    Q, _ = S.mixture(nq, D, 16, 3100 + D, comp_seed=3000 + D + B, scale="aniso")
    probe = S.random_probe_lists(nq, 64, 8, 3200 + D)
    k = 10
    ids, dists, cids, cest = gx.search(to_dev(Q), k, rerank_k=kp, probe=to_dev(probe), nprobe=8,
                                       precision="fp16", return_candidates=True)
    torch.cuda.synchronize()
    gid = cids.cpu().numpy()
    ge = cest.cpu().numpy().astype(np.float64)
    assert (gid >= 0).all()
    oest = oracle.estimate_rows(ox, Q, gid)
    bound = _bound(ox, Q, gid) + 2e-5 * (np.abs(oest) + 1e-3 * np.median(np.abs(oest)))
    viol = np.abs(ge - oest) > bound
    assert not viol.any(), f"{viol.sum()} estimates outside the FP16 bound"
    # ids: exact wherever the oracle's values are farther apart than the two
    # results' FP16 error bounds (reported), and the selected set is valid: for
    # every oracle top-k' id the GPU left out and every id it kept instead, the
    # two oracle estimates differ by no more than the sum of their bounds
    ref = oracle.search(ox, Q, k, kprime=kp + 1, probe=probe)
    rad = _bound(ox, Q, ref["cand_ids"]) + 2e-5 * np.abs(ref["cand_est"])
    frac = compare_topk_ids(gid, ref["cand_ids"], ref["cand_est"], what="fp16 candidates", radius=rad,
                            max_excluded=1.0)
    print(f"fp16 candidates: {frac:.3f} of slots within the error bound of a neighbour")
    b_gpu = bound
    for i in range(nq):
        top = dict(zip(ref["cand_ids"][i, :kp].tolist(), range(kp)))
        mine = dict(zip(gid[i].tolist(), range(kp)))
        missing = [j for o, j in top.items() if o not in mine]
        extra = [j for g, j in mine.items() if g not in top]
        assert len(missing) == len(extra)
        for jo in missing:
            for jg in extra:
                gap = oest[i, jg] - ref["cand_est"][i, jo]
                assert gap <= rad[i, jo] + b_gpu[i, jg] + 1e-9, (i, jo, jg, gap)
    # exact re-rank of the same candidate sets gives the oracle's top-k
    refr = oracle.search(ox, Q, k, kprime=kp, probe=probe)
    same = (np.sort(gid, 1) == np.sort(ref["cand_ids"][:, :kp], 1)).all(1)
    assert same.mean() > 0.5
    gi = ids.cpu().numpy()
    derr = assert_close_rel(dists.cpu().numpy()[same], refr["dists"][same], 1e-5, "re-ranked distances")
    compare_topk_ids(gi[same], refr["ids"][same], refr["dists"][same], 1.5 * max(derr, 1e-7), "re-ranked ids",
                     max_excluded=0.05)
    # every query (none exempt): the final top-k is the exact re-rank of the
    # candidate set the tensor-core scan selected
    frac = check_final_vs_own_candidates(X, Q, gid, gi, dists.cpu().numpy(), k)
    print(f"fp16 final top-{k}: {frac:.4f} of slots within a near-tie")


def test_tc_matches_fp32_recall(erq):
    X, P, gx, ox = _index(erq, 30000, 128, 4, 32, 3300)
    Q, _ = S.mixture(500, 128, 16, 3301, comp_seed=3300, scale="aniso")
    a_ids, _ = gx.search(to_dev(Q), 10, rerank_k=32, nprobe=6, precision="fp32")
    b_ids, _ = gx.search(to_dev(Q), 10, rerank_k=32, nprobe=6, precision="fp16")
    gt, _ = oracle.exact_knn(X, Q, 10)
    rec = lambda ids: np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.cpu().numpy(), gt)])
    ra, rb = rec(a_ids), rec(b_ids)
    assert rb >= ra - 0.005, (ra, rb)
    assert (a_ids == b_ids).float().mean().item() > 0.97


def test_tc_rejects_large_k(erq):
    X, P, gx, ox = _index(erq, 3000, 64, 4, 8, 3400)
    Q = to_dev(S.mixture(4, 64, 16, 3401, comp_seed=3400, scale="aniso")[0])
    with pytest.raises(erq.ErqError, match="tensor-core"):
        gx.search(Q, 10, rerank_k=129, nprobe=2, precision="fp16")


@pytest.mark.parametrize("qn,rr", [(32, 2048), (64, 4096), (128, 8192), (128, 256), (64, 512)])
def test_tc_scan_shapes_agree(erq, qn, rr):
    """Every work-item shape (queries per item = the MMA's N extent, rows per
    item) computes the same estimates and selects the same candidates: each
    item's list is a superset of its share of the query's top-k'."""
    X, P, gx, ox = _index(erq, 20000, 128, 5, 48, 3500)
    Q, _ = S.mixture(900, 128, 16, 3501, comp_seed=3500, scale="aniso")
    kw = dict(rerank_k=24, nprobe=12, precision="fp16", return_candidates=True)
    gx.set_scan_config(0, 0)
    ref = gx.search(to_dev(Q), 10, **kw)
    gx.set_scan_config(qn, rr)
    got = gx.search(to_dev(Q), 10, **kw)
    torch.cuda.synchronize()
    assert gx.scan_config() == (qn, rr)
    gx.set_scan_config(0, 0)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_autotune_picks_a_shape(erq):
    X, P, gx, ox = _index(erq, 20000, 128, 5, 48, 3600)
    Q = to_dev(S.mixture(1200, 128, 16, 3601, comp_seed=3600, scale="aniso")[0])
    ref = gx.search(Q, 10, rerank_k=20, nprobe=12, precision="fp16")
    best = gx.autotune(Q, 10, rerank_k=20, nprobe=12, precision="fp16", reps=2)
    assert best[0] in (32, 64, 128) and best[1] in (2048, 4096, 8192)
    got = gx.search(Q, 10, rerank_k=20, nprobe=12, precision="fp16")
    torch.cuda.synchronize()
    assert gx.scan_config() == best
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    with pytest.raises(erq.ErqError):
        gx.set_scan_config(48, 0)
    with pytest.raises(erq.ErqError):
        gx.set_scan_config(256, 0)
    with pytest.raises(erq.ErqError):
        gx.set_scan_config(0, 1000)


def _pack_reference(codes, off, B):
    """The packed scan layout written out from its definition (64-bit words
    [tile of 32 rows][block of 64 coordinates][B][32 rows], nibble halves for
    bits 0-3 when B >= 4, bit planes for the others), with numpy."""
    D = codes.shape[1]
    nkb = D // 64
    parts = []
    for c in range(len(off) - 1):
        blk = codes[off[c]:off[c + 1]]
        parts.append(np.concatenate([blk, np.zeros(((-len(blk)) % 32, D), np.uint8)]))
    U = np.concatenate(parts).astype(np.uint64)
    U = U.reshape(-1, 32, nkb, 64).transpose(0, 2, 1, 3)          # [tile, kb, r, 64 codes]
    W = np.zeros(U.shape[:3] + (B,), np.uint64)                   # [tile, kb, r, word]
    if B >= 4:
        half = np.zeros(U.shape[:3] + (8,), np.uint64)
        for h in range(8):
            for L in range(4):
                byte = (U[..., 8 * h + L] & 15) | ((U[..., 8 * h + 4 + L] & 15) << 4)
                half[..., h] |= byte << (8 * L)
        for w in range(4):
            W[..., w] = half[..., 2 * w] | (half[..., 2 * w + 1] << 32)
    for b in range(4 if B >= 4 else 0, B):
        half = np.zeros(U.shape[:3] + (2,), np.uint64)
        for m in range(16):
            for L in range(4):
                bit = (U[..., 4 * m + L] >> b) & 1
                half[..., m >> 3] |= bit << (8 * L + (m & 7))
        W[..., b] = half[..., 0] | (half[..., 1] << 32)
    return np.ascontiguousarray(W.transpose(0, 1, 3, 2)).view(np.uint8).ravel()   # [tile, kb, word, r]


@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_packed_scan_layout_bit_exact(erq, B):
    """The scan's packed copy holds exactly the index's codes, B bits each."""
    X, lab = S.mixture(3000, 128, 8, 3700 + B, scale="aniso")
    assign = S.kmeans_assign(X, 7, 3, 3701)
    P = S.random_orthogonal(128, 3702)
    gx = erq.build_index(to_dev(X), to_dev(P), B, 7, assign=to_dev(assign))
    codes = gx.export("codes").numpy()
    off = gx.export("list_offsets").numpy()
    got = gx.export("packed_codes").numpy()
    ref = _pack_reference(codes, off, B)
    assert got.shape == ref.shape and got.size == int(((off[1:] - off[:-1] + 31) // 32 * 32).sum()) * 128 * B // 8
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("B", [1, 2, 6, 8, 9])
def test_tc_scan_every_code_width(erq, B):
    """Estimates from the packed codes stay within the FP16 query-rounding
    bound for code widths the larger tests do not cover."""
    X, P, gx, ox = _index(erq, 8000, 128, B, 16, 3800 + B)
    Q, _ = S.mixture(300, 128, 16, 3801, comp_seed=3800 + B, scale="aniso")
    probe = S.random_probe_lists(300, 16, 4, 3802)
    ids, dists, cids, cest = gx.search(to_dev(Q), 10, rerank_k=24, probe=to_dev(probe), nprobe=4,
                                       precision="fp16", return_candidates=True)
    torch.cuda.synchronize()
    gid = cids.cpu().numpy()
    assert (gid >= 0).all()
    oest = oracle.estimate_rows(ox, Q, gid)
    bound = _bound(ox, Q, gid) + 2e-5 * (np.abs(oest) + 1e-3 * np.median(np.abs(oest)))
    viol = np.abs(cest.cpu().numpy().astype(np.float64) - oest) > bound
    assert not viol.any(), f"{viol.sum()} estimates outside the FP16 bound"


def _bound_fp8(ox, Q, ids):
    """Per-result bound of the e4m3 query rounding: every q'_i / s is rounded to
    the nearest e4m3 value (relative 2^-4, or absolute 2^-10 in the subnormal
    range), s = 2^(floor(log2 max|q'|) - 7) per query (taken twice as large here
    to cover the FP32 maximum landing on the other side of a power of two)."""
    B = ox["B"]
    qp = Q.astype(np.float64) @ ox["P"].astype(np.float64)
    s = 2.0 ** (np.floor(np.log2(np.abs(qp).max(1))) - 6)
    _, f_res = oracle.stored_factors(ox["stats"])
    rows = ox["row_of"][np.maximum(ids, 0)]
    y2 = np.abs(2.0 * ox["codes"][rows].astype(np.float64) - (2 ** B - 1))   # [nq, k, D]
    t = np.einsum("qkd,qd->qk", y2, np.abs(qp)) * 2.0 ** -4 + y2.sum(-1) * (s[:, None] * 2.0 ** -10)
    return 0.5 * np.abs(f_res[rows]).astype(np.float64) * t


@pytest.mark.parametrize("D,B,kp", [(128, 4, 32), (960, 4, 24), (128, 2, 100), (192, 3, 32),
                                    (128, 5, 32), (192, 7, 24), (256, 8, 100), (128, 6, 32), (960, 7, 32)])
def test_fp8_scan_within_e4m3_bound(erq, D, B, kp):
    """kind::f8f6f4 scan (e4m3 queries; B <= 4: e4m3 codes, 128 coordinates
    per stage, D = 960 and 192 ending in half a stage; B = 5..8: codes split
    into 16 hc + lc, 64 coordinates per stage): every candidate estimate lies
    within the query-rounding bound of the oracle's exact estimate, the
    selected set is valid, and the re-ranked top-10 equals the exact re-rank of
    the same candidates."""
    X, P, gx, ox = _index(erq, 12000, D, B, 32, 3900 + D + B)
    Q, _ = S.mixture(400, D, 16, 3901 + D, comp_seed=3900 + D + B, scale="aniso")
    probe = S.random_probe_lists(400, 32, 6, 3902 + D)
    ids, dists, cids, cest = gx.search(to_dev(Q), 10, rerank_k=kp, probe=to_dev(probe), nprobe=6,
                                       precision="fp8", return_candidates=True)
    torch.cuda.synchronize()
    gid = cids.cpu().numpy()
    assert (gid >= 0).all()
    oest = oracle.estimate_rows(ox, Q, gid)
    bound = _bound_fp8(ox, Q, gid) + 2e-5 * (np.abs(oest) + 1e-3 * np.median(np.abs(oest)))
    viol = np.abs(cest.cpu().numpy().astype(np.float64) - oest) > bound
    assert not viol.any(), f"{viol.sum()} estimates outside the e4m3 bound"
    # the selected set is valid: for every oracle top-k' id the GPU left out
    # and every id it kept instead, the two oracle estimates differ by no more
    # than the sum of their e4m3 bounds
    ref = oracle.search(ox, Q, 10, kprime=kp, probe=probe)
    rad = _bound_fp8(ox, Q, ref["cand_ids"]) + 2e-5 * np.abs(ref["cand_est"])
    for i in range(len(Q)):
        top = dict(zip(ref["cand_ids"][i].tolist(), range(kp)))
        mine = dict(zip(gid[i].tolist(), range(kp)))
        missing = [j for o, j in top.items() if o not in mine]
        extra = [j for g, j in mine.items() if g not in top]
        assert len(missing) == len(extra)
        for jo in missing:
            for jg in extra:
                gap = oest[i, jg] - ref["cand_est"][i, jo]
                assert gap <= rad[i, jo] + bound[i, jg] + 1e-9, (i, jo, jg, gap)
    # every query's final top-10 is the exact re-rank of its own candidate set
    frac = check_final_vs_own_candidates(X, Q, gid, ids.cpu().numpy(), dists.cpu().numpy(), 10)
    print(f"fp8 final top-10: {frac:.4f} of slots within a near-tie")


def test_fp8_recall_close_to_fp32(erq):
    X, P, gx, ox = _index(erq, 30000, 128, 4, 32, 4000)
    Q, _ = S.mixture(500, 128, 16, 4001, comp_seed=4000, scale="aniso")
    a_ids, _ = gx.search(to_dev(Q), 10, rerank_k=40, nprobe=6, precision="fp32")
    b_ids, _ = gx.search(to_dev(Q), 10, rerank_k=40, nprobe=6, precision="fp8")
    gt, _ = oracle.exact_knn(X, Q, 10)
    rec = lambda ids: np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.cpu().numpy(), gt)])
    ra, rb = rec(a_ids), rec(b_ids)
    assert rb >= ra - 0.01, (ra, rb)


def test_fp8_rejects_nine_bit_codes(erq):
    """B = 9: the split parts would need 5 bits (16 hc with |hc| <= 31), which
    e4m3 does not hold exactly; the search refuses instead of rounding codes."""
    X, P, gx, ox = _index(erq, 3000, 128, 9, 8, 4150)
    Q = to_dev(S.mixture(4, 128, 16, 4151, comp_seed=4150, scale="aniso")[0])
    with pytest.raises(erq.ErqError, match="B <= 8"):
        gx.search(Q, 10, rerank_k=20, nprobe=2, precision="fp8")


def test_fp8_split_recall_close_to_fp32(erq):
    """B = 7 (the precision workload's code width) in the split e4m3 form:
    recall@10 after the exact re-rank stays within 0.01 of the FP32 scan's."""
    X, P, gx, ox = _index(erq, 30000, 256, 7, 32, 4100)
    Q, _ = S.mixture(500, 256, 16, 4101, comp_seed=4100, scale="aniso")
    a_ids, _ = gx.search(to_dev(Q), 10, rerank_k=40, nprobe=6, precision="fp32")
    b_ids, _ = gx.search(to_dev(Q), 10, rerank_k=40, nprobe=6, precision="fp8")
    gt, _ = oracle.exact_knn(X, Q, 10)
    rec = lambda ids: np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.cpu().numpy(), gt)])
    ra, rb = rec(a_ids), rec(b_ids)
    assert rb >= ra - 0.01, (ra, rb)
