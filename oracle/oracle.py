"""Python driver of the FP64 C oracle (erq_oracle.c).

TEST INFRASTRUCTURE ONLY.  Follows arXiv 2409.09913:

* ``centroids`` / ``rotate``   -- local centring (Section 5.1) and o' = P^{-1}(o_r - c)
  (Section 3.3 workflow), readings R1/R2 of erq_oracle.c.
* ``quantize``                  -- Algorithm 1 (Section 3.1).
* ``build_index``               -- IVF index: clusters from an input assignment
  (Section 4.1), codes and per-vector factors (Section 5.1 metrics paragraph).
* ``search``                    -- probe, Eq. 3.3 + Eq. (eq:dis to ip) estimates, top-k',
  exact re-rank, top-k; or the same for inner products (reading R9: Section 7
  defers the inner-product metric to RaBitQ's estimator).
* ``rerank``                    -- exact re-rank of given candidate sets (FP64, numpy).
* ``estimate_rows`` / ``backward`` -- estimated distances of given pairs and their
  gradient w.r.t. the raw query.
* ``brute_force_quantize``      -- exhaustive argmax of Eq. 3.2 (optimization) over the
  whole grid G, for tiny D and B (pin for Algorithm 1).
* ``two_stage_search``          -- Section 4.2: estimates from the most significant bits
  (the 1-bit RaBitQ code, Lemma 2.1 estimator and bound) prune the probed rows,
  Eq. 4.2 completes the survivors' estimates; numpy, FP64.
"""
from __future__ import annotations

import ctypes as ct
import functools
import itertools

import numpy as np

from . import build as _build

__all__ = [
    "lib", "centroids", "rotate", "quantize", "build_index", "search", "estimate_rows",
    "backward", "rerank", "centroid_dists", "brute_force_quantize", "exact_knn", "num_threads",
    "stored_factors", "two_stage_search", "two_stage_rows",
]

_lib = None
_P = np.ctypeslib.ndpointer
_f32 = _P(np.float32, flags="C_CONTIGUOUS")
_f64 = _P(np.float64, flags="C_CONTIGUOUS")
_i32 = _P(np.int32, flags="C_CONTIGUOUS")
_i64 = _P(np.int64, flags="C_CONTIGUOUS")
_u16 = _P(np.uint16, flags="C_CONTIGUOUS")


class _Opt:
    """ndpointer that also accepts None."""

    def __init__(self, dtype):
        self.base = _P(dtype, flags="C_CONTIGUOUS")

    def from_param(self, obj):
        if obj is None:
            return None
        return self.base.from_param(obj)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        L.orc_centroids.argtypes = [_f32, ct.c_int64, ct.c_int, _i32, ct.c_int, _f32]
        L.orc_rotate.argtypes = [_f32, _Opt(np.float32), _Opt(np.int32), ct.c_int64, ct.c_int, _f32, _f32]
        L.orc_quantize_batch.argtypes = [_f32, ct.c_int64, ct.c_int, ct.c_int, _u16, _f64]
        L.orc_search.argtypes = [ct.c_int, ct.c_int, ct.c_int, _f32, _f32, _i64, _i64, _u16, _f64, _f32,
                                 _f64, ct.c_int64, _i32, _Opt(np.int32), ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                                 _i64, _f64, _Opt(np.int64), _Opt(np.float64), _Opt(np.int32)]
        L.orc_centroid_dists.argtypes = [_f32, ct.c_int, ct.c_int, _f64, ct.c_int64, _f64]
        L.orc_estimate_rows.argtypes = [ct.c_int, ct.c_int, _f32, _f32, _u16, _f64, _f64, ct.c_int64, ct.c_int,
                                        _i64, _i32, ct.c_int, _f64]
        L.orc_backward.argtypes = [ct.c_int, ct.c_int, _f32, _f32, _u16, _f64, _f64, ct.c_int64, ct.c_int,
                                   _i64, _i32, _f64, ct.c_int, _f64]
        L.orc_num_threads.restype = ct.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def centroids(X, assign, nlist):
    X = _c32(X)
    C = np.empty((nlist, X.shape[1]), np.float32)
    lib().orc_centroids(X, X.shape[0], X.shape[1], np.ascontiguousarray(assign, np.int32), nlist, C)
    return C


def rotate(X, P, C=None, assign=None):
    """Rows of fl32(P^T (x - c)) accumulated in FP64 (reading R2)."""
    X = _c32(X)
    out = np.empty_like(X)
    lib().orc_rotate(X, None if C is None else _c32(C),
                     None if assign is None else np.ascontiguousarray(assign, np.int32),
                     X.shape[0], X.shape[1], _c32(P), out)
    return out


def quantize(Rp, B):
    """Algorithm 1 on each row.  Returns (codes uint16 [n,d], stats float64 [n,5]);
    stats = (<ybar,|o'|>, ||ybar||^2, v_max, ||o'||^2, events)."""
    Rp = _c32(np.atleast_2d(Rp))
    n, d = Rp.shape
    codes = np.empty((n, d), np.uint16)
    stats = np.empty((n, 5), np.float64)
    lib().orc_quantize_batch(Rp, n, d, int(B), codes, stats)
    return codes, stats


def stored_factors(stats):
    """The two FP32 per-vector factors held by an index, from the FP64 stats:
    f_add = ||o'||^2 and f_res = -2 ||o'||^2 / <ybar, |o'|> (0 when o' = 0), so that
    est = f_add + ||q_r - c||^2 + f_res * <ybar, P^T (q_r - c)>  (Eq. 3.3 with
    Eq. (eq:dis to ip), ||ybar|| cancelling)."""
    ip, nr2 = stats[:, 0], stats[:, 3]
    f_add = nr2.astype(np.float32)
    with np.errstate(divide="ignore", invalid="ignore"):
        f_res = np.where(nr2 > 0, (-2.0 * nr2) / ip, 0.0).astype(np.float32)
    return f_add, f_res


def build_index(X, P, assign, nlist, B, centroids_in=None):
    """IVF + extended-RaBitQ index, all in FP64 (Sections 3.3, 4.1).

    Centroids are the cluster means (reading R1) unless ``centroids_in`` is
    given (e.g. c = 0, the un-centred setting of Section 2.2)."""
    X = _c32(X)
    assign = np.ascontiguousarray(assign, np.int32)
    n, d = X.shape
    C = centroids(X, assign, nlist) if centroids_in is None else _c32(centroids_in)
    Rp = rotate(X, P, C, assign)
    order = np.argsort(assign, kind="stable").astype(np.int64)
    counts = np.bincount(assign, minlength=nlist).astype(np.int64)
    list_off = np.zeros(nlist + 1, np.int64)
    list_off[1:] = np.cumsum(counts)
    codes, stats = quantize(Rp[order], B)
    row_of = np.empty(n, np.int64)
    row_of[order] = np.arange(n, dtype=np.int64)
    return dict(d=d, B=int(B), nlist=int(nlist), P=_c32(P), C=C, Cp=rotate(C, P), list_off=list_off,
                list_ids=order, codes=codes, stats=stats, X=X, assign=assign, row_of=row_of,
                Rp=Rp)


def _q64(Q):
    return np.ascontiguousarray(np.atleast_2d(Q), dtype=np.float64)


def search(ix, Q, k, kprime=0, nprobe=None, probe=None, metric="l2"):
    """Batched search; returns dict(ids, dists, cand_ids, cand_est, probe).

    ``nprobe``: int or per-query array; ``probe``: optional explicit [nq, maxp]
    probe lists (then nprobe per query defaults to maxp).  ``metric``: "l2"
    (squared distances, ascending) or "ip" (inner products, descending; reading
    R9 of erq_oracle.c)."""
    if metric not in ("l2", "ip"):
        raise ValueError(metric)
    Q = _q64(Q)
    nq = Q.shape[0]
    if probe is not None:
        probe = np.ascontiguousarray(probe, np.int32)
        maxp = probe.shape[1]
        npr = np.full(nq, maxp, np.int32) if nprobe is None else np.broadcast_to(
            np.asarray(nprobe, np.int32), (nq,)).copy()
    else:
        npr = np.broadcast_to(np.asarray(ix["nlist"] if nprobe is None else nprobe, np.int32), (nq,)).copy()
        maxp = int(npr.max()) if nq else 1
    kp = kprime if kprime > 0 else k
    ids = np.empty((nq, k), np.int64)
    dists = np.empty((nq, k), np.float64)
    cand_ids = np.empty((nq, kp), np.int64)
    cand_est = np.empty((nq, kp), np.float64)
    probe_out = np.full((nq, maxp), -1, np.int32)
    lib().orc_search(ix["d"], ix["B"], ix["nlist"], ix["P"], ix["C"], ix["list_off"], ix["list_ids"],
                     ix["codes"], ix["stats"], ix["X"], Q, nq, np.ascontiguousarray(npr), probe, maxp,
                     int(kprime), int(k), 1 if metric == "ip" else 0, ids, dists, cand_ids, cand_est, probe_out)
    return dict(ids=ids, dists=dists, cand_ids=cand_ids, cand_est=cand_est, probe=probe_out)


def _rows_and_clusters(ix, ids):
    ids = np.asarray(ids, np.int64)
    rows = np.where(ids >= 0, ix["row_of"][np.maximum(ids, 0)], -1).astype(np.int64)
    cl = np.repeat(np.arange(ix["nlist"], dtype=np.int32), np.diff(ix["list_off"]))
    return np.ascontiguousarray(rows), np.ascontiguousarray(cl)


def estimate_rows(ix, Q, ids, metric="l2"):
    """Estimated squared distance (metric "l2") or inner product (metric "ip",
    reading R9) of query i to each original id in ids[i, :]."""
    if metric not in ("l2", "ip"):
        raise ValueError(metric)
    Q = _q64(Q)
    ids = np.atleast_2d(ids)
    rows, cl = _rows_and_clusters(ix, ids)
    out = np.empty(ids.shape, np.float64)
    lib().orc_estimate_rows(ix["d"], ix["B"], ix["P"], ix["C"], ix["codes"], ix["stats"], Q, Q.shape[0],
                            ids.shape[1], rows, cl, 1 if metric == "ip" else 0, out)
    return out


def backward(ix, Q, ids, g, metric="l2"):
    """sum_j g[i,j] * d est(q_i, ids[i,j]) / d q_i  (FP64); est is the estimated
    squared distance (metric "l2") or inner product (metric "ip")."""
    if metric not in ("l2", "ip"):
        raise ValueError(metric)
    Q = _q64(Q)
    ids = np.atleast_2d(ids)
    rows, cl = _rows_and_clusters(ix, ids)
    out = np.empty(Q.shape, np.float64)
    lib().orc_backward(ix["d"], ix["B"], ix["P"], ix["C"], ix["codes"], ix["stats"], Q, Q.shape[0],
                       ids.shape[1], rows, cl, np.ascontiguousarray(g, np.float64), 1 if metric == "ip" else 0, out)
    return out


def rerank(X, Q, cand_ids, k, metric="l2"):
    """Exact re-rank of given candidate sets (the last step of the search):
    for query i, the FP64 squared distance ||x_j - q_i||^2 (metric "l2") or
    inner product <x_j, q_i> (metric "ip") of every candidate id j >= 0 in
    cand_ids[i], ordered by (distance, id) ascending (inner products: by
    (-<x_j, q_i>, id)), first k kept.  Returns (ids int64 [nq, k], values
    float64 [nq, k]) with -1 / +inf (ip: -inf) where fewer than k candidates
    exist.  Written out from the definition with numpy, independent of the C
    file."""
    if metric not in ("l2", "ip"):
        raise ValueError(metric)
    X = np.asarray(X)
    Q = _q64(Q)
    cand_ids = np.atleast_2d(np.asarray(cand_ids, np.int64))
    nq = Q.shape[0]
    ids = np.full((nq, k), -1, np.int64)
    vals = np.full((nq, k), np.inf if metric == "l2" else -np.inf, np.float64)
    for i in range(nq):
        c = np.unique(cand_ids[i][cand_ids[i] >= 0])
        if len(c) == 0:
            continue
        x = X[c].astype(np.float64)
        v = ((x - Q[i]) ** 2).sum(1) if metric == "l2" else -(x @ Q[i])
        o = np.lexsort((c, v))[:k]
        ids[i, :len(o)] = c[o]
        vals[i, :len(o)] = v[o] if metric == "l2" else -v[o]
    return ids, vals


def centroid_dists(C, Q):
    Q = _q64(Q)
    C = _c32(C)
    out = np.empty((Q.shape[0], C.shape[0]), np.float64)
    lib().orc_centroid_dists(C, C.shape[0], C.shape[1], Q, Q.shape[0], out)
    return out


def exact_knn(X, Q, k):
    """Exact k nearest rows by FP64 squared distance, ties by id (ground truth)."""
    X64 = np.asarray(X, np.float64)
    ids = np.empty((len(Q), k), np.int64)
    dd = np.empty((len(Q), k), np.float64)
    for i, q in enumerate(np.asarray(Q, np.float64)):
        d2 = ((X64 - q) ** 2).sum(1)
        o = np.lexsort((np.arange(len(X64)), d2))[:k]
        ids[i], dd[i] = o, d2[o]
    return ids, dd


@functools.lru_cache(maxsize=16)
def _grid(d, B):
    levels = np.arange(2 ** B, dtype=np.float64) - (2 ** B - 1) / 2.0   # Eq. (equ:shift)
    grid = np.array(list(itertools.product(levels, repeat=d)), dtype=np.float64)
    return grid, np.linalg.norm(grid, axis=1)


def brute_force_quantize(op, B):
    """argmax over the whole grid G of <y/||y||, o'> (Eq. 3.2, optimization) by
    enumeration of all 2^(B*D) grid vectors.  Returns (best cosine, list of
    ybar_u codes that reach it within 4 ulp)."""
    op = np.asarray(op, np.float64)
    grid, gnorm = _grid(op.shape[0], int(B))
    cos = grid @ op / gnorm / np.linalg.norm(op)
    best = cos.max()
    tol = 4 * np.spacing(abs(best))
    hits = grid[cos >= best - tol] + (2 ** B - 1) / 2.0
    return best, hits.astype(np.int64)


def two_stage_rows(ix, q, c, rows, eps0):
    """Per-row quantities of the two-stage search for one query q and one
    cluster c (stored rows ``rows`` of that cluster), FP64:

    * est1: Lemma 2.1's estimate from the row's most significant bits, which
      form the 1-bit RaBitQ code of the same residual (Section 4.2): with
      xbar = 2 msb - 1 (+-1 per coordinate), obar_0 = P xbar / sqrt(D) and the
      unit residual o, <o, q^> ~ <obar_0, q^> / <obar_0, o>, where
      <obar_0, o> = sum_i |o'_i| / (sqrt(D) ||o'||);
    * bound: Lemma 2.1's error bound carried to the squared distance
      ||o'||^2 + ||q_r - c||^2 - 2 ||o'|| ||q_r - c|| <o, q^>:
      2 ||o'|| ||q_r - c|| sqrt(1 - a^2) / a * eps0 / sqrt(D - 1), a = <obar_0, o>;
    * est: the full B-bit estimate (Eq. 3.3, Eq. (eq:dis to ip)) with
      <ybar_u, q'> assembled by Eq. 4.2 from the stage-1 product of the MSB
      code and the product of the remaining bits;
    * ip_msb: <msb, q'> (q' the unit rotated residual query), reused by Eq. 4.2.
    Rows with o' = 0 (reading R8) estimate ||q_r - c||^2 with bound 0."""
    d, B = ix["d"], ix["B"]
    codes = ix["codes"][rows].astype(np.float64)
    st = ix["stats"][rows]
    qn = np.asarray(q, np.float64) - ix["C"][c].astype(np.float64)
    qc = np.sqrt(qn @ qn)
    if qc > 0:
        qn = qn / qc
    qp = qn @ ix["P"].astype(np.float64)                 # P^{-1} q^ (P orthogonal)
    sum_qp = qp.sum()
    msb = np.floor(codes / 2 ** (B - 1))                 # the MSB plane, 0/1
    last = codes - 2 ** (B - 1) * msb                    # the remaining B-1 bits
    ip_msb = msb @ qp
    ipu = 2 ** (B - 1) * ip_msb + last @ qp              # Eq. 4.2
    op = ix["Rp"][ix["list_ids"][rows]].astype(np.float64)
    nr2 = (op * op).sum(1)
    nr = np.sqrt(nr2)
    pos = nr2 > 0
    safe = np.where(pos, nr, 1.0)
    a = np.abs(op).sum(1) / (np.sqrt(d) * safe)          # <obar_0, o>
    # 1-bit estimate: ||ybar_1|| <obar_0, q^> = <msb, q'> - sum q' / 2 with ||ybar_1|| = sqrt(D)/2
    ip1 = np.where(pos, (ip_msb - 0.5 * sum_qp) / (0.5 * np.sqrt(d) * np.where(pos, a, 1.0)), 0.0)
    est1 = nr2 + qc * qc - 2.0 * nr * qc * ip1
    with np.errstate(divide="ignore", invalid="ignore"):
        bound = np.where(pos, 2.0 * nr * qc * np.sqrt(np.maximum(1.0 - a * a, 0.0)) / np.where(pos, a, 1.0)
                         * eps0 / np.sqrt(d - 1), 0.0)
    # full estimate from the stored stats (as the search): ||ybar|| <obar, q^> * 1/(||ybar|| <o, obar>)
    obar_q = ipu - 0.5 * (2 ** B - 1) * sum_qp
    o_obar = np.where(pos, st[:, 2] / safe, 1.0)
    inv = np.where(pos, 1.0 / (np.sqrt(st[:, 1]) * o_obar), 0.0)
    est = nr2 + qc * qc - 2.0 * nr * qc * obar_q * inv
    return dict(est1=est1, bound=bound, est=est, ip_msb=ip_msb)


def two_stage_search(ix, Q, k, kprime, nprobe=None, probe=None, eps0=1.9):
    """Two-stage (MSB-first) search of Section 4.2, FP64 with numpy (metric l2).

    Per query: the probe of ``search``; stage 1 gives every probed row its
    1-bit estimate est1 and Lemma 2.1 bound (two_stage_rows).  Pruning rule
    (reading): tau = the k'-th smallest upper bound est1 + bound over the
    query's probed rows (+inf with fewer than k' rows); when every bound holds,
    at least k' rows have a true distance <= tau, so no row of the true top-k'
    has est1 - bound > tau, and only those rows are dropped.  Stage 2: the
    survivors' full estimates (Eq. 4.2), their top-k' by (estimate, id), the
    exact re-rank and top-k as in ``search``.  eps0 = inf keeps every row
    (the single-stage search); eps0 = 0 keeps the k' smallest est1.

    Returns dict(ids, dists, cand_ids, cand_est, tau, survivors, rows, probe)."""
    Q = _q64(Q)
    nq = Q.shape[0]
    kp = kprime if kprime > 0 else k
    pr = search(ix, Q, k, kprime, nprobe=nprobe, probe=probe)["probe"]
    cand_ids = np.full((nq, kp), -1, np.int64)
    cand_est = np.full((nq, kp), np.inf)
    tau = np.full(nq, np.inf)
    surv = np.zeros(nq, np.int64)
    nrows = np.zeros(nq, np.int64)
    for i in range(nq):
        ids, e1, bd, est = [], [], [], []
        for c in pr[i]:
            if c < 0:
                continue
            rows = np.arange(ix["list_off"][c], ix["list_off"][c + 1])
            if len(rows) == 0:
                continue
            r = two_stage_rows(ix, Q[i], c, rows, eps0)
            ids.append(ix["list_ids"][rows])
            e1.append(r["est1"])
            bd.append(r["bound"])
            est.append(r["est"])
        if not ids:
            continue
        ids, e1, bd, est = map(np.concatenate, (ids, e1, bd, est))
        nrows[i] = len(ids)
        ub = e1 + bd
        if len(ub) >= kp:
            tau[i] = np.sort(ub)[kp - 1]
        keep = ~(e1 - bd > tau[i])
        surv[i] = keep.sum()
        o = np.lexsort((ids[keep], est[keep]))[:kp]
        cand_ids[i, :len(o)] = ids[keep][o]
        cand_est[i, :len(o)] = est[keep][o]
    rids, rd = rerank(ix["X"], Q, cand_ids, k)
    return dict(ids=rids, dists=rd, cand_ids=cand_ids, cand_est=cand_est, tau=tau, survivors=surv, rows=nrows,
                probe=pr)
