"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test ties the oracle to something other than itself: hand-worked
examples (tests/golden), exhaustive enumeration on tiny inputs, lemmas of the
paper, closed-form limits, statistical properties the paper states, and
library routines for the plain linear-algebra steps.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", _golden()["alg1"], ids=lambda c: f"B{c['B']}-{c['op']}")
def test_alg1_hand_examples(case):
    """Hand-enumerated argmax of Eq. 3.2 (tests/golden/hand_examples.json)."""
    op = np.array(case["op"], np.float32)
    codes, st = oracle.quantize(op, case["B"])
    assert codes[0].tolist() == case["code"]
    expect = eval(case["vmax_over_norm"], {"math": math})
    assert st[0, 2] / math.sqrt(st[0, 3]) == pytest.approx(expect, rel=1e-6)


@pytest.mark.parametrize("B", [1, 2, 3])
@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_alg1_equals_brute_force(B, d):
    """Algorithm 1 returns the maximum-cosine grid vector of Eq. 3.2 (optimization),
    checked against enumeration of all 2^(B*D) vectors of G."""
    if B * d > 18:
        pytest.skip("grid too large")
    n = 120 if B * d >= 18 else (200 if B * d > 12 else 400)
    for kind, seed in (("gauss", 11), ("ties", 12), ("sparse", 13)):
        R = S.random_rotated_residuals(n, d, seed + 100 * d + B, kind=kind)
        codes, st = oracle.quantize(R, B)
        for i in range(n):
            if not np.any(R[i]):
                continue
            best, hits = oracle.brute_force_quantize(R[i], B)
            v = st[i, 2] / math.sqrt(st[i, 3])
            assert v == pytest.approx(best, rel=1e-13, abs=1e-15), (kind, R[i], codes[i])
            assert any((h == codes[i]).all() for h in hits), (kind, R[i], codes[i], hits)


@pytest.mark.parametrize("d,B", [(1, 9), (2, 9), (1, 10), (2, 10)])
def test_alg1_wide_codes_equal_brute_force(d, B):
    """B = 9 and 10 (Section 5.1 evaluates B up to 9, Table 4 times B up to
    10): Algorithm 1 against enumeration of all 2^(B D) grid vectors (512 to
    1,048,576)."""
    n = 60 if d == 2 else 200
    for kind, seed in (("gauss", 15), ("ties", 16), ("sparse", 17)):
        R = S.random_rotated_residuals(n, d, seed + 100 * d + 1000 * (B - 9), kind=kind)
        codes, st = oracle.quantize(R, B)
        assert codes.max() <= 2 ** B - 1
        for i in range(n):
            if not np.any(R[i]):
                continue
            best, hits = oracle.brute_force_quantize(R[i], B)
            v = st[i, 2] / math.sqrt(st[i, 3])
            assert v == pytest.approx(best, rel=1e-13, abs=1e-15), (kind, R[i], codes[i])
            assert any((h == codes[i]).all() for h in hits), (kind, R[i], codes[i], hits)


def test_alg1_b1_is_rabitq_sign_code():
    """B = 1: the codebook is RaBitQ's (Section 3.1) -- code = sign bits of o',
    <obar,o> = sum|o'| / (sqrt(D) ||o'||) (Section 2.2)."""
    R = S.random_rotated_residuals(500, 128, 5, kind="sparse")
    codes, st = oracle.quantize(R, 1)
    assert (codes == (R >= 0).astype(np.uint8)).all()
    r64 = R.astype(np.float64)
    expect = np.abs(r64).sum(1) / math.sqrt(128) / np.linalg.norm(r64, axis=1)
    np.testing.assert_allclose(st[:, 2] / np.sqrt(st[:, 3]), expect, rtol=1e-13)
    assert (st[:, 4] == 0).all()          # no critical values when B = 1


@pytest.mark.parametrize("B", [2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_alg1_msb_is_sign_and_event_count(B):
    """Section 4.2: the most significant bits of ybar_u form the RaBitQ code of
    o'.  Section 3.1: each non-zero coordinate has 2^(B-1)-1 critical values."""
    R = S.random_rotated_residuals(300, 64, 20 + B, kind="sparse")
    codes, st = oracle.quantize(R, B)
    assert ((codes >> (B - 1)) == (R >= 0)).all()
    assert codes.max() <= 2 ** B - 1
    nz = (R != 0).sum(1)
    assert (st[:, 4] == nz * (2 ** (B - 1) - 1)).all()


@pytest.mark.parametrize("B", [2, 3, 5, 7, 9, 10])
def test_lemma_3_1_nearest_grid_point(B):
    """Lemma 3.1 with the proof's t = ||ybar||^2 / <o', ybar>: ybar is a
    nearest point of G to t*o' (G is a product set, so coordinate-wise)."""
    R = S.random_rotated_residuals(200, 96, 30 + B)
    codes, st = oracle.quantize(R, B)
    levels = np.arange(2 ** B) - (2 ** B - 1) / 2.0
    for i in range(len(R)):
        o = R[i].astype(np.float64)
        y = codes[i].astype(np.float64) - (2 ** B - 1) / 2.0
        t = (y @ y) / (o @ y)
        dist_y = np.abs(t * o - y)
        dist_best = np.abs(t * o[:, None] - levels[None, :]).min(1)
        assert (dist_y <= dist_best + 1e-9).all()


@pytest.mark.parametrize("B", [1, 3, 6])
def test_lemma_b1_identity(B):
    """Lemma B.1: 1 - <o,obar>^2 = min_{t>0,y in G} ||o' - t y||^2, reached by
    ybar at t = <o', ybar/||ybar||>/||ybar||; any other grid vector does no
    better (checked on random one-coordinate moves of ybar)."""
    g = S.rng(40 + B)
    R = S.random_rotated_residuals(100, 48, 41 + B)
    codes, st = oracle.quantize(R, B)
    for i in range(len(R)):
        o = R[i].astype(np.float64)
        o /= np.linalg.norm(o)
        y = codes[i].astype(np.float64) - (2 ** B - 1) / 2.0
        o_obar = o @ y / np.linalg.norm(y)
        t = o_obar / np.linalg.norm(y)
        lhs = 1.0 - o_obar ** 2
        assert np.sum((o - t * y) ** 2) == pytest.approx(lhs, abs=1e-12)
        assert o_obar == pytest.approx(st[i, 2] / math.sqrt(st[i, 3]), rel=1e-12)
        for _ in range(20):
            y2 = y.copy()
            j = g.integers(len(y))
            y2[j] = g.choice(np.arange(2 ** B) - (2 ** B - 1) / 2.0)
            t2 = (o @ y2) / (y2 @ y2)
            if t2 > 0:
                assert np.sum((o - t2 * y2) ** 2) >= lhs - 1e-12


def test_b1_concentration_and_growth_with_b():
    """Section 2.2: for B = 1, <obar,o> concentrates near 0.8 (the limit for
    uniform o is sqrt(2/pi) = 0.7979); footnote of Section 3.1: <obar,o>
    increases with B."""
    R = S.random_rotated_residuals(2000, 1024, 50)
    means = []
    for B in (1, 2, 3, 4):
        _, st = oracle.quantize(R, B)
        c = st[:, 2] / np.sqrt(st[:, 3])
        means.append(c.mean())
        if B == 1:
            assert abs(c.mean() - math.sqrt(2 / math.pi)) < 2e-3
            assert c.std() < 0.01
    assert all(b > a for a, b in zip(means, means[1:]))


# --------------------------------------------------------------------------
# Linear-algebra steps (library routines as independent references)
# --------------------------------------------------------------------------
def test_rotation_matches_library_matmul():
    """o' = P^{-1} o = P^T o for orthogonal P (Section 3.3 workflow)."""
    P = S.random_orthogonal(64, 3)
    assert np.abs(P.astype(np.float64) @ P.T.astype(np.float64) - np.eye(64)).max() < 1e-6
    X, lab = S.mixture(500, 64, 4, 3)
    C = oracle.centroids(X, lab, 4)
    Rp = oracle.rotate(X, P, C, lab)
    resid = (X.astype(np.float64) - C[lab].astype(np.float64)).astype(np.float32).astype(np.float64)
    ref = P.astype(np.float64).T @ resid.T
    err = np.abs(Rp.astype(np.float64) - ref.T)
    assert (err <= np.spacing(np.abs(Rp)) * 1.0 + 1e-30).all()
    np.testing.assert_allclose(np.linalg.norm(Rp, axis=1), np.linalg.norm(resid, axis=1), rtol=1e-5)


def test_centroids_match_library_mean():
    X, lab = S.mixture(3000, 32, 8, 4)
    C = oracle.centroids(X, lab, 8)
    for j in range(8):
        ref = X[lab == j].astype(np.float64).mean(0)
        assert (np.abs(C[j] - ref) <= np.spacing(np.abs(C[j])) + 1e-30).all()


# --------------------------------------------------------------------------
# Estimator
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", _golden()["estimator"], ids=lambda c: f"B{c['B']}")
def test_estimator_hand_examples(case):
    o = np.array([case["o"]], np.float32)
    q = np.array([case["q"]], np.float64)
    ix = oracle.build_index(o, np.eye(2, dtype=np.float32), np.zeros(1, np.int32), 1, case["B"],
                            centroids_in=np.zeros((1, 2), np.float32))
    est = oracle.estimate_rows(ix, q, np.array([[0]]))[0, 0]
    assert est == pytest.approx(eval(case["est"]), rel=1e-6)
    ex = oracle.search(ix, q, 1, kprime=1, nprobe=1)
    assert ex["dists"][0, 0] == pytest.approx(eval(case["true"]), rel=1e-6)


def _unit_pairs(n, d, seed):
    g = S.rng(seed)
    o = g.standard_normal((n, d))
    q = g.standard_normal((n, d))
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return o.astype(np.float32), q


def _ip_estimates(o, q, B, P):
    """Estimated <o,q> of unit vectors from the oracle's distance estimate
    (c = 0, so est = 2 - 2 <o,q>_est by Eq. eq:dis to ip)."""
    n, d = o.shape
    ix = oracle.build_index(o, P, np.zeros(n, np.int32), 1, B, centroids_in=np.zeros((1, d), np.float32))
    est = oracle.estimate_rows(ix, q, np.arange(n, dtype=np.int64)[:, None])[:, 0]
    on = np.linalg.norm(o.astype(np.float64), axis=1)
    qn = np.linalg.norm(q, axis=1)
    return (on ** 2 + qn ** 2 - est) / (2 * on * qn)


@pytest.mark.parametrize("B", [2, 3])
def test_estimator_unbiased_over_rotations(B):
    """Lemma 2.1 (kept by the new codebook, Section 3.2): averaged over random
    orthogonal P, the estimate of <o,q> equals <o,q>."""
    d, trials = 16, 1500
    o, q = _unit_pairs(1, d, 60 + B)
    true = float(o[0].astype(np.float64) @ q[0])
    vals = []
    for t in range(trials):
        P = S.random_orthogonal(d, 1000 + t)
        vals.append(_ip_estimates(o, q, B, P)[0])
    vals = np.array(vals)
    se = vals.std() / math.sqrt(trials)
    assert abs(vals.mean() - true) < 4 * se + 1e-12
    # and the estimate is not trivially exact
    assert vals.std() > 1e-4


def test_error_decays_as_empirical_formula():
    """Section 3.3 remark / Section 5.2.6: the 99.9% quantile of the absolute
    error of the unit-vector inner-product estimate follows 5.75 * 2^-B / sqrt(D).
    The constant is a fitted one ("the curves match well"), so the quantile may
    sit a little above it: allowed up to 1.25x.  The shape is pinned tighter:
    the quantile halves per extra bit and scales as D^-1/2."""
    q999 = {}
    for d, n in ((64, 20000), (256, 8000)):
        o, q = _unit_pairs(n, d, 70 + d)
        P = S.random_orthogonal(d, 71)
        true = (o.astype(np.float64) * q).sum(1)
        for B in range(1, 10):
            err = np.abs(_ip_estimates(o, q, B, P) - true)
            q999[d, B] = np.quantile(err, 0.999)
            assert q999[d, B] < 1.25 * 5.75 * 2.0 ** -B / math.sqrt(d), (d, B, q999[d, B])
        slope = np.polyfit(np.arange(1, 10), np.log2([q999[d, B] for B in range(1, 10)]), 1)[0]
        assert -1.1 < slope < -0.9, slope
    d_slope = np.mean([np.log2(q999[256, B] / q999[64, B]) / 2 for B in range(1, 10)])
    assert -0.6 < d_slope < -0.4, d_slope


def test_unbiased_regression_slope_one():
    """Section 5.2.5 (Fig. 6): estimated vs true squared distances, normalised
    by the maximum, fit a line of slope 1 and intercept 0."""
    X, lab = S.mixture(4000, 128, 4, 80, scale="aniso")
    Q, _ = S.mixture(8, 128, 4, 81, comp_seed=80, scale="aniso")
    P = S.random_orthogonal(128, 82)
    ix = oracle.build_index(X, P, np.zeros(len(X), np.int32), 1, 2)
    ids = np.tile(np.arange(len(X)), (len(Q), 1))
    est = oracle.estimate_rows(ix, Q, ids).ravel()
    true = ((X[None, :, :].astype(np.float64) - Q[:, None, :]) ** 2).sum(-1).ravel()
    m = true.max()
    slope, icpt = np.polyfit(true / m, est / m, 1)
    assert abs(slope - 1) < 0.01 and abs(icpt) < 0.01


def test_high_b_estimate_close_to_exact():
    X, lab = S.mixture(2000, 96, 4, 90)
    Q, _ = S.mixture(4, 96, 4, 91, comp_seed=90)
    P = S.random_orthogonal(96, 92)
    ix = oracle.build_index(X, P, lab, 4, 8)
    ids = np.tile(np.arange(len(X)), (len(Q), 1))
    est = oracle.estimate_rows(ix, Q, ids)
    true = ((X[None].astype(np.float64) - Q[:, None].astype(np.float64)) ** 2).sum(-1)
    assert np.mean(np.abs(est - true) / true) < 2e-3


def test_zero_residual_reading():
    """Reading R8: o_r = c gives estimate ||q_r - c||^2."""
    X = np.array([[1.0, 2.0, 3.0, 4.0]], np.float32)
    ix = oracle.build_index(X, S.random_orthogonal(4, 1), np.zeros(1, np.int32), 1, 3)
    q = np.array([[0.5, 0.0, 1.0, -1.0]])
    est = oracle.estimate_rows(ix, q, np.array([[0]]))[0, 0]
    assert est == pytest.approx(((X[0] - q[0]) ** 2).sum(), rel=1e-12)


# --------------------------------------------------------------------------
# Search, top-k, backward
# --------------------------------------------------------------------------
def test_search_full_rerank_is_exact_knn():
    """Probing every cluster and re-ranking every candidate with exact
    distances must return the exact k nearest neighbours (ties by id)."""
    X, lab = S.mixture(1500, 32, 6, 100)
    X[10] = X[11]                      # an exact tie
    Q = np.concatenate([X[10:11], S.mixture(5, 32, 6, 101, comp_seed=100)[0]])
    ix = oracle.build_index(X, S.random_orthogonal(32, 102), lab, 6, 3)
    res = oracle.search(ix, Q, 10, kprime=len(X), nprobe=6)
    gt, gd = oracle.exact_knn(X, Q, 10)
    np.testing.assert_array_equal(res["ids"], gt)
    np.testing.assert_allclose(res["dists"], gd, rtol=1e-12)
    assert res["ids"][0, 0] == 10 and res["ids"][0, 1] == 11


def test_rerank_hand_example_and_ties():
    """Exact re-rank of a given candidate set, worked by hand: points at
    squared distances 4, 1, 1, 9 and 0 from q = 0 (ids 7, 3, 5, 2, 9; id 9
    not a candidate, id 3 listed twice, one empty slot): (3, 1), (5, 1) with
    the tie by lower id, then (7, 4), then (2, 9); a fifth slot stays empty."""
    X = np.zeros((10, 2), np.float32)
    X[7], X[3], X[5], X[2], X[9] = (2, 0), (0, 1), (-1, 0), (0, -3), (0, 0)
    ids, vals = oracle.rerank(X, np.zeros((1, 2)), np.array([[7, 3, 5, -1, 2, 3]]), 5)
    np.testing.assert_array_equal(ids[0], [3, 5, 7, 2, -1])
    np.testing.assert_array_equal(vals[0], [1.0, 1.0, 4.0, 9.0, np.inf])
    ids, vals = oracle.rerank(X, np.array([[1.0, 1.0]]), np.array([[7, 3, 5, 2]]), 2, metric="ip")
    np.testing.assert_array_equal(ids[0], [7, 3])          # <x, q> = 2, 1, -1, -3
    np.testing.assert_array_equal(vals[0], [2.0, 1.0])


def test_rerank_matches_the_c_search():
    """The numpy re-rank of the C search's own candidate sets gives the C
    search's re-ranked ids and distances (two independent codings of the
    exact re-rank), for both metrics."""
    X, lab = S.mixture(3000, 48, 8, 104)
    ix = oracle.build_index(X, S.random_orthogonal(48, 105), lab, 8, 4)
    Q = S.mixture(30, 48, 8, 106, comp_seed=104)[0]
    for metric in ("l2", "ip"):
        res = oracle.search(ix, Q, 10, kprime=40, nprobe=3, metric=metric)
        ids, vals = oracle.rerank(X, Q, res["cand_ids"], 10, metric=metric)
        np.testing.assert_array_equal(ids, res["ids"])
        np.testing.assert_allclose(vals, res["dists"], rtol=1e-12)


def test_search_probe_is_nearest_centroids():
    X, lab = S.mixture(2000, 16, 10, 110)
    ix = oracle.build_index(X, S.random_orthogonal(16, 111), lab, 10, 2)
    Q = S.mixture(20, 16, 10, 112, comp_seed=110)[0].astype(np.float64)
    res = oracle.search(ix, Q, 5, nprobe=3)
    cd = ((Q[:, None, :] - ix["C"][None].astype(np.float64)) ** 2).sum(-1)
    ref = np.argsort(cd, axis=1, kind="stable")[:, :3]
    np.testing.assert_array_equal(res["probe"], ref)


def test_search_estimates_rank_like_exact():
    """B = 7 with IVF and no re-ranking recovers most true neighbours
    (Section 5.2.2 reports >99% recall at 7 bits on real data)."""
    X, lab = S.mixture(6000, 64, 8, 120, scale="aniso")
    Q = S.mixture(30, 64, 8, 121, comp_seed=120, scale="aniso")[0]
    ix = oracle.build_index(X, S.random_orthogonal(64, 122), lab, 8, 7)
    res = oracle.search(ix, Q, 10, kprime=0, nprobe=8)
    gt, _ = oracle.exact_knn(X, Q, 10)
    recall = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(res["ids"], gt)])
    assert recall > 0.9


def test_backward_matches_finite_differences():
    """The gradient of the estimated scores w.r.t. the raw query equals
    central finite differences (h = 1e-3, FP64) of the oracle's estimate."""
    X, lab = S.mixture(300, 16, 3, 130)
    ix = oracle.build_index(X, S.random_orthogonal(16, 131), lab, 3, 4)
    Q = S.mixture(3, 16, 3, 132, comp_seed=130)[0].astype(np.float64)
    ids = np.stack([S.rng(133 + i).choice(300, 7, replace=False) for i in range(3)])
    g = S.normal((3, 7), 134).astype(np.float64)
    grad = oracle.backward(ix, Q, ids, g)
    h = 1e-3
    fd = np.zeros_like(Q)
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        fp = (oracle.estimate_rows(ix, Q + e, ids) * g).sum(1)
        fm = (oracle.estimate_rows(ix, Q - e, ids) * g).sum(1)
        fd[:, k] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-7, atol=1e-7)


def test_stored_factors_reproduce_estimate():
    """The two stored floats per vector (Section 5.1 metrics paragraph) with
    <ybar, P^T(q_r - c)> reproduce the estimate (library matmul for P^T)."""
    X, lab = S.mixture(400, 32, 2, 140)
    P = S.random_orthogonal(32, 141)
    ix = oracle.build_index(X, P, lab, 2, 5)
    Q = S.mixture(3, 32, 2, 142, comp_seed=140)[0].astype(np.float64)
    f_add, f_res = oracle.stored_factors(ix["stats"])
    rows = np.arange(400)
    cl = np.repeat(np.arange(2), np.diff(ix["list_off"]))
    ids = ix["list_ids"][rows]
    est = oracle.estimate_rows(ix, Q, np.tile(ids, (3, 1)))
    for i in range(3):
        qt = (Q[i][None, :] - ix["C"][cl].astype(np.float64)) @ P.astype(np.float64)
        ybar = ix["codes"].astype(np.float64) - (2 ** 5 - 1) / 2
        ref = f_add + ((Q[i][None, :] - ix["C"][cl]) ** 2).sum(1) + f_res * (ybar * qt).sum(1)
        np.testing.assert_allclose(est[i], ref, rtol=2e-6)


# --------------------------------------------------------------------------
# Inner-product metric (reading R9 of erq_oracle.c)
# --------------------------------------------------------------------------
def _ip_est_single(o, c, q, B, P):
    """Estimated <o, q> of one stored vector o (centroid c) through the
    oracle's inner-product search (one row, one cluster, no re-rank)."""
    d = o.shape[0]
    ix = oracle.build_index(o[None].astype(np.float32), P, np.zeros(1, np.int32), 1, B,
                            centroids_in=c[None].astype(np.float32))
    res = oracle.search(ix, q[None], 1, kprime=0, nprobe=1, metric="ip")
    return res["dists"][0, 0], res["cand_est"][0, 0]


def test_ip_search_full_rerank_is_exact_mips():
    """Probing every cluster and re-ranking every candidate by the exact inner
    product returns the exact top-k by <o, q> (ties by lower id), reported
    with their inner products in decreasing order."""
    X, lab = S.mixture(1500, 32, 6, 150)
    X[20] = X[21] = 4.0 * X[21]                       # an exact tie, near the top for most queries
    Q = np.concatenate([X[20:21], S.mixture(5, 32, 6, 151, comp_seed=150)[0]]).astype(np.float64)
    ix = oracle.build_index(X, S.random_orthogonal(32, 152), lab, 6, 3)
    res = oracle.search(ix, Q, 10, kprime=len(X), nprobe=6, metric="ip")
    ip = Q @ X.astype(np.float64).T
    ref = np.stack([np.lexsort((np.arange(len(X)), -row))[:10] for row in ip])
    np.testing.assert_array_equal(res["ids"], ref)
    np.testing.assert_allclose(res["dists"], np.take_along_axis(ip, ref, 1), rtol=1e-12)
    assert (np.diff(res["dists"], axis=1) <= 0).all()
    assert res["ids"][0, 0] == 20 and res["ids"][0, 1] == 21      # <x, x> is the largest for q = x here


def test_ip_probe_is_largest_inner_products():
    X, lab = S.mixture(2000, 16, 10, 160)
    ix = oracle.build_index(X, S.random_orthogonal(16, 161), lab, 10, 2)
    Q = S.mixture(20, 16, 10, 162, comp_seed=160)[0].astype(np.float64)
    res = oracle.search(ix, Q, 5, nprobe=3, metric="ip")
    ref = np.argsort(-(Q @ ix["C"].astype(np.float64).T), axis=1, kind="stable")[:, :3]
    np.testing.assert_array_equal(res["probe"], ref)


@pytest.mark.parametrize("B", [2, 4, 7])
def test_ip_estimate_exact_for_residual_on_the_grid(B):
    """When the rotated residual is a multiple of a grid vector ybar (Eq.
    equ:shift), <obar, o> = 1 and the estimate equals the exact inner product:
    this ties together the <c, q> term, the ||o_r - c|| ||q_r|| scale, the
    (2^B - 1)/2 shift and the factor 1/(||ybar|| <obar, o>)."""
    d = 12
    g = S.rng(170 + B)
    perm = g.permutation(d)
    P = np.zeros((d, d), np.float32)
    P[perm, np.arange(d)] = g.choice([-1.0, 1.0], d)           # signed permutation: exact in FP32
    c = (g.integers(-8, 9, d) / 4.0).astype(np.float32)
    for t in range(5):
        yu = g.integers(0, 2 ** B, d)
        ybar = yu - (2 ** B - 1) / 2.0
        o_rot = 0.5 * ybar                                       # on the grid direction, exact in FP32
        o = (c.astype(np.float64) + P.astype(np.float64) @ o_rot).astype(np.float32)
        assert np.array_equal(P.astype(np.float64).T @ (o.astype(np.float64) - c), o_rot)
        q = g.standard_normal(d) * 3.0
        est, cand = _ip_est_single(o, c, q, B, P)
        true = float(o.astype(np.float64) @ q)
        scale = abs(float(c @ q)) + np.linalg.norm(o_rot) * np.linalg.norm(q)
        assert abs(est - true) <= 1e-12 * scale, (B, t, est, true)
        assert est == cand


def test_ip_zero_residual_gives_centroid_term():
    """o_r = c: the estimate is <c, q_r> (reading R8 carried to R9)."""
    c = np.array([1.0, -2.0, 0.5, 3.0], np.float32)
    q = np.array([0.25, 1.0, -2.0, 0.75])
    est, _ = _ip_est_single(c.copy(), c, q, 3, S.random_orthogonal(4, 3))
    assert est == pytest.approx(float(c.astype(np.float64) @ q), rel=1e-12)


@pytest.mark.parametrize("B", [2, 3])
def test_ip_estimator_unbiased_over_rotations(B):
    """Lemma 2.1 carried to R9: averaged over random orthogonal P, the estimated
    <o_r, q_r> equals the exact one (nonzero centroid, unnormalised vectors)."""
    d, trials = 16, 1500
    g = S.rng(180 + B)
    o = g.standard_normal(d).astype(np.float32)
    c = (0.5 * g.standard_normal(d)).astype(np.float32)
    q = g.standard_normal(d) * 2.0
    true = float(o.astype(np.float64) @ q)
    vals = np.array([_ip_est_single(o, c, q, B, S.random_orthogonal(d, 2000 + t))[0] for t in range(trials)])
    se = vals.std() / math.sqrt(trials)
    assert abs(vals.mean() - true) < 4 * se + 1e-12
    assert vals.std() > 1e-4


def test_ip_estimate_rows_agree_with_search():
    """The pairwise inner-product estimate is the one the search ranks by."""
    X, lab = S.mixture(800, 24, 4, 190)
    ix = oracle.build_index(X, S.random_orthogonal(24, 191), lab, 4, 4)
    Q = S.mixture(6, 24, 4, 192, comp_seed=190)[0].astype(np.float64)
    res = oracle.search(ix, Q, 5, kprime=0, nprobe=4, metric="ip")
    est = oracle.estimate_rows(ix, Q, res["cand_ids"], metric="ip")
    np.testing.assert_allclose(est, res["cand_est"], rtol=0, atol=0)
    assert (np.diff(res["cand_est"], axis=1) <= 0).all()


def test_ip_backward_matches_finite_differences():
    """The gradient of the estimated inner products w.r.t. the raw query equals
    central finite differences (h = 1e-3, FP64) of the oracle's estimate; the
    estimate is linear in q_r, so the differences are exact up to rounding."""
    X, lab = S.mixture(300, 16, 3, 195)
    ix = oracle.build_index(X, S.random_orthogonal(16, 196), lab, 3, 4)
    Q = S.mixture(3, 16, 3, 197, comp_seed=195)[0].astype(np.float64)
    ids = np.stack([S.rng(198 + i).choice(300, 7, replace=False) for i in range(3)])
    g = S.normal((3, 7), 199).astype(np.float64)
    grad = oracle.backward(ix, Q, ids, g, metric="ip")
    h = 1e-3
    fd = np.zeros_like(Q)
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        fp = (oracle.estimate_rows(ix, Q + e, ids, metric="ip") * g).sum(1)
        fm = (oracle.estimate_rows(ix, Q - e, ids, metric="ip") * g).sum(1)
        fd[:, k] = (fp - fm) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("case", _golden()["inner_product"], ids=lambda c: f"B{c['B']}-c{c['c']}")
def test_ip_estimator_hand_examples(case):
    """Hand-derived inner-product estimates (tests/golden), P = I."""
    o = np.array(case["o"], np.float32)
    c = np.array(case["c"], np.float32)
    q = np.array(case["q"], np.float64)
    est, _ = _ip_est_single(o, c, q, case["B"], np.eye(2, dtype=np.float32))
    assert est == pytest.approx(eval(case["est"]), rel=1e-6)
    X = o[None].astype(np.float32)
    ix = oracle.build_index(X, np.eye(2, dtype=np.float32), np.zeros(1, np.int32), 1, case["B"],
                            centroids_in=c[None])
    ex = oracle.search(ix, q[None], 1, kprime=1, nprobe=1, metric="ip")
    assert ex["dists"][0, 0] == pytest.approx(eval(case["true"]), rel=1e-6)
