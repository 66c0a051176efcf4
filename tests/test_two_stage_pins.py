"""Pins of the oracle's two-stage (MSB-first) search, Section 4.2.

The stage-1 quantities are tied to the C oracle's own 1-bit index (the paper's
observation that the most significant bits are the original RaBitQ code), the
stage-2 estimate to the C oracle's full B-bit estimate, the two limits of the
pruning rule to the single-stage searches, and the bound to Lemma 2.1's
statement on random rotations.
"""
import numpy as np
import pytest

import oracle
import synthetic as S


def _setup(n=4000, d=64, nlist=8, B=5, seed=0):
    X, _ = S.mixture(n, d, 8, seed, scale="aniso")
    assign = S.kmeans_assign(X, nlist, 3, seed + 1)
    P = S.random_orthogonal(d, seed + 2)
    ix = oracle.build_index(X, P, assign, nlist, B)
    Q, _ = S.mixture(24, d, 8, seed + 3, comp_seed=seed, scale="aniso")
    return X, P, assign, ix, Q


@pytest.mark.parametrize("B", [2, 3, 5, 8, 9])
def test_msb_plane_is_the_one_bit_code(B):
    """Section 4.2: the most significant bits of the B-bit code are the 1-bit
    RaBitQ code of the same rotated residual, and the stage-1 factor
    <obar_0, o> = sum |o'_i| / (sqrt(D) ||o'||) is the 1-bit encoder's v_max / ||o'||."""
    X, P, assign, ix, Q = _setup(B=B, seed=10 + B)
    Rs = ix["Rp"][ix["list_ids"]]
    c1, st1 = oracle.quantize(Rs, 1)
    assert np.array_equal(ix["codes"] >> (B - 1), c1)
    op = Rs.astype(np.float64)
    a = np.abs(op).sum(1) / (np.sqrt(op.shape[1]) * np.sqrt((op * op).sum(1)))
    np.testing.assert_allclose(a, st1[:, 2] / np.sqrt(st1[:, 3]), rtol=1e-12)


def test_stage_one_is_the_one_bit_estimate():
    """est1 equals the C oracle's estimate in a 1-bit index of the same data,
    centroids and rotation (Lemma 2.1's estimator)."""
    X, P, assign, ix, Q = _setup(seed=20)
    ix1 = oracle.build_index(X, P, assign, ix["nlist"], 1, centroids_in=ix["C"])
    for i in range(4):
        for c in range(ix["nlist"]):
            rows = np.arange(ix["list_off"][c], ix["list_off"][c + 1])
            r = oracle.two_stage_rows(ix, Q[i], c, rows, 1.9)
            ref = oracle.estimate_rows(ix1, Q[i:i + 1], ix["list_ids"][rows][None, :])[0]
            np.testing.assert_allclose(r["est1"], ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("B", [1, 3, 5, 7, 9])
def test_stage_two_is_the_full_estimate(B):
    """Eq. 4.2 (MSB product reused, remaining bits added) gives the C oracle's
    full B-bit estimate."""
    X, P, assign, ix, Q = _setup(B=B, seed=30 + B)
    for i in range(4):
        for c in range(ix["nlist"]):
            rows = np.arange(ix["list_off"][c], ix["list_off"][c + 1])
            r = oracle.two_stage_rows(ix, Q[i], c, rows, 1.9)
            ref = oracle.estimate_rows(ix, Q[i:i + 1], ix["list_ids"][rows][None, :])[0]
            np.testing.assert_allclose(r["est"], ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())


def test_no_pruning_limit_is_the_single_stage_search():
    """eps0 = inf keeps every row: candidates and answer of ``search``."""
    X, P, assign, ix, Q = _setup(seed=40)
    a = oracle.search(ix, Q, 10, kprime=40, nprobe=3)
    b = oracle.two_stage_search(ix, Q, 10, 40, nprobe=3, eps0=np.inf)
    assert np.array_equal(a["cand_ids"], b["cand_ids"])
    np.testing.assert_allclose(b["cand_est"], a["cand_est"], rtol=1e-10)
    assert np.array_equal(a["ids"], b["ids"])
    assert (b["survivors"] == b["rows"]).all()


def test_zero_bound_limit_keeps_the_one_bit_top_kprime():
    """eps0 = 0: the bound vanishes, tau is the k'-th smallest est1 and the
    survivors are the 1-bit index's top-k' (the C oracle's 1-bit search)."""
    X, P, assign, ix, Q = _setup(seed=50)
    ix1 = oracle.build_index(X, P, assign, ix["nlist"], 1, centroids_in=ix["C"])
    r1 = oracle.search(ix1, Q, 10, kprime=30, nprobe=3)
    b = oracle.two_stage_search(ix, Q, 10, 30, nprobe=3, eps0=0.0)
    assert (b["survivors"] == 30).all()
    for i in range(len(Q)):
        assert set(b["cand_ids"][i].tolist()) == set(r1["cand_ids"][i].tolist())


def test_bound_holds_with_lemma_probability_and_prunes_no_true_neighbour():
    """Lemma 2.1: over random rotations the stage-1 error exceeds the bound
    with probability at most exp(-c0 eps0^2).  The measured violation rates
    fall as a normal tail in eps0 (the bound at eps0 = 1 is about one standard
    deviation of the error): about 0.3 at 1, 0.04 at 2, below 1e-3 at 4.
    Where every bound of a query holds (eps0 = 4), the rows of its true
    top-k' (exact distances over the probed rows) all survive the pruning."""
    d, B, nlist = 96, 4, 6
    X, _ = S.mixture(3000, d, 8, 60, scale="aniso")
    assign = S.kmeans_assign(X, nlist, 3, 61)
    Q, _ = S.mixture(12, d, 8, 62, comp_seed=60, scale="aniso")
    rates = {0.5: [], 1.0: [], 2.0: [], 4.0: []}
    kept_checked = 0
    for rot in range(6):
        P = S.random_orthogonal(d, 100 + rot)
        ix = oracle.build_index(X, P, assign, nlist, B)
        res = oracle.two_stage_search(ix, Q, 10, 25, nprobe=2, eps0=4.0)
        for i in range(len(Q)):
            ids, e1, bd, ex = [], [], [], []
            for c in res["probe"][i]:
                rows = np.arange(ix["list_off"][c], ix["list_off"][c + 1])
                r = oracle.two_stage_rows(ix, Q[i], c, rows, 1.0)
                gid = ix["list_ids"][rows]
                ids.append(gid)
                e1.append(r["est1"])
                bd.append(r["bound"])
                ex.append(((X[gid].astype(np.float64) - Q[i]) ** 2).sum(1))
            ids, e1, bd, ex = map(np.concatenate, (ids, e1, bd, ex))
            for eps in rates:
                rates[eps].append(np.mean(np.abs(e1 - ex) > eps * bd))
            if not (np.abs(e1 - ex) <= 4.0 * bd).all():
                continue
            kept_checked += 1
            true_top = ids[np.lexsort((ids, ex))[:25]]
            ub = e1 + 4.0 * bd
            tau = np.sort(ub)[24]
            survivors = set(ids[~(e1 - 4.0 * bd > tau)].tolist())
            assert set(true_top.tolist()) <= survivors
            assert res["survivors"][i] == len(survivors)
    r = {e: float(np.mean(v)) for e, v in rates.items()}
    assert r[0.5] > r[1.0] > r[2.0] > r[4.0], r
    assert 0.2 < r[1.0] < 0.4 and 0.015 < r[2.0] < 0.07 and r[4.0] < 1e-3, r
    for e, v in r.items():
        assert v <= np.exp(-0.4 * e * e), (e, v)
    assert kept_checked >= 40
