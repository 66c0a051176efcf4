"""Helpers shared by the GPU parity tests (comparison rules written once)."""
import numpy as np
import pytest
import torch

# Tolerance of the FP32 GPU path against the FP64 oracle (relative, with an
# absolute floor proportional to the typical magnitude of the row).
FP32_RTOL = 1e-5


@pytest.fixture(scope="session")
def erq():
    from paper_2409_09913_gb300 import build, erq as _erq
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return _erq


def dev():
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def assert_close_rel(got, ref, rtol=FP32_RTOL, what="values"):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    fin = np.isfinite(ref)
    assert (np.isfinite(got) == fin).all(), f"{what}: finiteness differs"
    scale = np.abs(ref[fin]) + 1e-3 * np.median(np.abs(ref[fin])) if fin.any() else 1.0
    err = np.abs(got[fin] - ref[fin]) / scale
    assert err.max(initial=0.0) <= rtol, f"{what}: max rel err {err.max():.3e} > {rtol}"
    return err.max(initial=0.0)


def check_final_vs_own_candidates(X, Q, cand_ids, ids, dists, k, metric="l2", what="re-ranked", max_excluded=0.01):
    """The search's final output for EVERY query against the exact FP64
    re-rank (oracle.rerank) of the candidate set the GPU itself selected:
    distances within 1e-5 relative (inner products: within 1e-5 * ||q|| *
    max ||x||, absolute), ids bit-exact at every slot not decided by a near-tie
    of that size.  Returns the fraction of excluded slots."""
    import oracle
    cand = np.asarray(cand_ids)
    got_i = np.asarray(ids)
    got_d = np.asarray(dists, np.float64)
    ref_i, ref_d = oracle.rerank(X, Q, cand, k + 1, metric=metric)
    if metric == "l2":
        derr = assert_close_rel(got_d, ref_d[:, :k], FP32_RTOL, f"{what} distances")
        radius = None
        tol = 1.5 * max(derr, 1e-7)
    else:
        Q64 = np.asarray(Q, np.float64)
        fin = np.isfinite(ref_d[:, :k])
        assert (np.isfinite(got_d) == fin).all(), f"{what}: finiteness differs"
        scale = np.linalg.norm(Q64, axis=1, keepdims=True) * np.linalg.norm(np.asarray(X, np.float64), axis=1).max()
        err = np.abs(got_d - ref_d[:, :k])[fin] / np.broadcast_to(scale, got_d.shape)[fin]
        assert err.max(initial=0.0) <= FP32_RTOL, f"{what} inner products: max err {err.max():.3e}"
        radius = np.broadcast_to(1.5 * max(err.max(initial=0.0), 1e-7) * scale, ref_d.shape)
        tol = None
    return compare_topk_ids(got_i, ref_i, ref_d, tol, f"{what} ids", max_excluded=max_excluded, radius=radius)


def compare_topk_ids(got_ids, ref_ids, ref_vals, tol=None, what="ids", max_excluded=0.02, radius=None):
    """Ids must match bit-exactly wherever the oracle's ranking is not decided
    by a near-tie.  ``ref_ids``/``ref_vals`` may carry one extra column (the
    oracle's (k+1)-th entry) so that ties across the cut are detected.  Slot j
    of query i is compared unless the oracle's value j lies within the sum of
    the two slots' error radii of value j-1 or j+1: the radius of a slot is
    ``radius[i, j]`` (absolute, per result) when given, else ``tol * |value|``.
    Returns the fraction of excluded slots, which must stay below max_excluded."""
    got_ids = np.asarray(got_ids)
    ref_ids = np.asarray(ref_ids)
    v = np.asarray(ref_vals, np.float64)
    r = np.asarray(radius, np.float64) if radius is not None else tol * np.abs(v)
    nq, k = got_ids.shape
    excluded = 0
    for i in range(nq):
        vi, ri = v[i], r[i]
        fin = np.isfinite(vi)
        for j in range(k):
            if not fin[j]:
                assert got_ids[i, j] == -1, f"{what}: query {i} slot {j} should be empty"
                continue
            near = (j > 0 and abs(vi[j] - vi[j - 1]) <= ri[j] + ri[j - 1]) or \
                   (j + 1 < len(vi) and fin[j + 1] and abs(vi[j + 1] - vi[j]) <= ri[j] + ri[j + 1])
            if near:
                excluded += 1
                continue
            assert got_ids[i, j] == ref_ids[i, j], f"{what}: query {i} slot {j}: {got_ids[i, j]} != {ref_ids[i, j]}"
    frac = excluded / max(1, nq * k)
    assert frac <= max_excluded, f"{what}: too many near-tie exclusions ({frac:.3f})"
    return frac
