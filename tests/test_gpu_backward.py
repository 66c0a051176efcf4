"""GPU backward (gradient of estimated scores w.r.t. the query) against the
FP64 oracle gradient and FP64 central finite differences (h = 1e-3)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _setup(erq, N=3000, D=128, B=4, nlist=6, nq=9, nc=25, seed=2000):
    X, lab = S.mixture(N, D, nlist, seed, scale="aniso")
    P = S.random_orthogonal(D, seed + 1)
    gx = erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(lab))
    ox = oracle.build_index(X, P, lab, nlist, B)
    Q, _ = S.mixture(nq, D, nlist, seed + 2, comp_seed=seed, scale="aniso")
    ids = np.stack([S.rng(seed + 3 + i).choice(N, nc, replace=False) for i in range(nq)]).astype(np.int64)
    g = S.normal((nq, nc), seed + 50)
    return X, P, gx, ox, Q, ids, g


def test_backward_matches_oracle_and_fd(erq):
    X, P, gx, ox, Q, ids, g = _setup(erq)
    ids[2, 4] = -1                              # ignored candidate
    got = gx.search_backward(to_dev(Q), to_dev(ids), to_dev(g)).cpu().numpy().astype(np.float64)
    ref = oracle.backward(ox, Q, ids, g.astype(np.float64))
    scale = np.abs(ref).max(1, keepdims=True)
    assert (np.abs(got - ref) / scale).max() < 2e-5
    # FP64 central differences of the oracle's estimated scores at the same query
    h = 1e-3
    Q64 = Q.astype(np.float64)
    for k in range(0, Q.shape[1], 17):
        e = np.zeros(Q.shape[1])
        e[k] = h
        fp = (np.nan_to_num(oracle.estimate_rows(ox, Q64 + e, ids)) * g).sum(1)
        fm = (np.nan_to_num(oracle.estimate_rows(ox, Q64 - e, ids)) * g).sum(1)
        fd = (fp - fm) / (2 * h)
        assert np.abs(got[:, k] - fd).max() / scale.max() < 2e-5


def test_autograd_function(erq):
    from paper_2409_09913_gb300.autograd import EstimatedScores, search_scores
    X, P, gx, ox, Q, ids, g = _setup(erq, seed=2100)
    Qt = to_dev(Q).requires_grad_(True)
    scores = EstimatedScores.apply(Qt, gx, to_dev(ids))
    (scores * to_dev(g)).sum().backward()
    ref = oracle.backward(ox, Q, ids, g.astype(np.float64))
    got = Qt.grad.cpu().numpy()
    assert (np.abs(got - ref) / np.abs(ref).max()).max() < 2e-5
    # the search-then-score helper returns the estimated top-k of the search
    Qt2 = to_dev(Q).requires_grad_(True)
    sid, sc = search_scores(gx, Qt2, 5, nprobe=3)
    sc.sum().backward()
    assert Qt2.grad.shape == Qt2.shape and torch.isfinite(Qt2.grad).all()
    assert sid.shape == (Q.shape[0], 5)


def test_backward_empty_candidates(erq):
    X, P, gx, ox, Q, ids, g = _setup(erq, nq=3, nc=4, seed=2200)
    ids[:] = -1
    got = gx.search_backward(to_dev(Q), to_dev(ids), to_dev(g)).cpu().numpy()
    assert np.all(got == 0)


def test_ip_estimate_and_backward_match_oracle(erq):
    """Inner-product metric: estimates <c, q_r> - (f_res/2) <ybar, P^T q_r> and
    their gradient c - (f_res/2) P ybar against the FP64 oracle (absolute
    tolerance scaled by ||q_r|| max ||o_r||, as inner products can be ~0)."""
    X, P, gx, ox, Q, ids, g = _setup(erq, seed=2300)
    ids[1, 3] = -1                              # ignored candidate
    est = gx.estimate(to_dev(Q), to_dev(ids), metric="ip").cpu().numpy().astype(np.float64)
    ref = oracle.estimate_rows(ox, Q, ids, metric="ip")
    assert np.isnan(est[1, 3]) and np.isnan(ref[1, 3])
    ok = ids >= 0
    sc = np.linalg.norm(Q.astype(np.float64), axis=1)[:, None] * np.linalg.norm(X.astype(np.float64), axis=1).max()
    assert (np.abs(est - ref)[ok] <= 1e-5 * np.broadcast_to(sc, est.shape)[ok]).all()
    got = gx.search_backward(to_dev(Q), to_dev(ids), to_dev(g), metric="ip").cpu().numpy().astype(np.float64)
    refg = oracle.backward(ox, Q, ids, g.astype(np.float64), metric="ip")
    scale = np.abs(refg).max(1, keepdims=True)
    assert (np.abs(got - refg) / scale).max() < 2e-5
    # autograd over the inner products
    from paper_2409_09913_gb300.autograd import EstimatedScores
    Qt = to_dev(Q).requires_grad_(True)
    (EstimatedScores.apply(Qt, gx, to_dev(ids), "ip").nan_to_num() * to_dev(g)).sum().backward()
    assert (np.abs(Qt.grad.cpu().numpy() - refg) / scale).max() < 2e-5
