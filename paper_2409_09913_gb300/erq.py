"""Thin Python binding of liberq.so (include/erq.h) -- argument marshalling only.

Every step of the search path runs in the library's CUDA kernels; this module
only checks tensor shapes/dtypes, passes device pointers and the current CUDA
stream, and turns error codes into exceptions.  It has no CPU fallback: if the
shared library is missing it raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liberq.so")

ERQ_OK, ERQ_EINVAL, ERQ_ENOMEM, ERQ_ECUDA, ERQ_ETIMEOUT, ERQ_EUNSUPPORTED, ERQ_EIO = range(7)
PREC = {"fp32": 0, "fp16": 1, "fp8": 2, "int8": 3}
METRIC = {"l2": 0, "ip": 1, "cos": 2}
FIELDS = {"centroids": 0, "rot_centroids": 1, "list_offsets": 2, "list_ids": 3, "codes": 4, "f_add": 5,
          "f_res": 6, "P": 7, "raw": 8, "packed_codes": 9}

# names of every entry point declared in include/erq.h
EXPORTS = ["erq_version", "erq_last_error", "erq_build_index", "erq_free_index", "erq_index_info_get",
           "erq_index_status", "erq_rotate", "erq_encode", "erq_search", "erq_search_host", "erq_estimate",
           "erq_search_backward", "erq_index_export", "erq_index_save", "erq_index_load", "erq_search_timing",
           "erq_kernel_launches", "erq_search_stats", "erq_search_backward_noalloc", "erq_search_timing_total",
           "erq_autotune", "erq_set_scan_config", "erq_scan_config", "erq_estimate_metric",
           "erq_search_backward_metric", "erq_merge_topk", "erq_rerank_ids", "erq_set_wait_limit",
           "erq_search_two_stage"]


class ErqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"erq error {code}: {msg}")
        self.code = code


class BuildParams(ct.Structure):
    _fields_ = [("B", ct.c_int32), ("nlist", ct.c_int32), ("P", ct.c_void_p), ("assign", ct.c_void_p),
                ("kmeans_iters", ct.c_int32), ("kmeans_sample", ct.c_int32), ("seed", ct.c_uint64),
                ("keep_raw", ct.c_int32), ("normalize", ct.c_int32), ("centroids", ct.c_void_p)]


class SearchParams(ct.Structure):
    _fields_ = [("k", ct.c_int32), ("rerank_k", ct.c_int32), ("nprobe", ct.c_int32), ("precision", ct.c_int32),
                ("nprobe_per_query", ct.c_void_p), ("probe", ct.c_void_p), ("probe_stride", ct.c_int32),
                ("flags", ct.c_int32), ("cand_ids", ct.c_void_p), ("cand_est", ct.c_void_p), ("metric", ct.c_int32)]


class IndexInfo(ct.Structure):
    _fields_ = [("N", ct.c_int64), ("D", ct.c_int32), ("B", ct.c_int32), ("nlist", ct.c_int32),
                ("keep_raw", ct.c_int32), ("max_list", ct.c_int64), ("device_bytes", ct.c_int64)]


_lib = None


def lib(path: str | None = None):
    """Load liberq.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    # ERQ_CHECKED=1 selects the build with device-side bound checks (liberq_checked.so)
    p = path or (LIB_PATH.replace("liberq.so", "liberq_checked.so") if os.environ.get("ERQ_CHECKED") == "1"
                 else LIB_PATH)
    if not os.path.exists(p):
        raise RuntimeError(f"liberq.so not found at {p}: run __graft_entry__.build() (or "
                           f"python -m paper_2409_09913_gb300.build) first; there is no CPU fallback")
    L = ct.CDLL(p)
    vp, i64, i32 = ct.c_void_p, ct.c_int64, ct.c_int32
    L.erq_version.restype = ct.c_char_p
    L.erq_last_error.restype = ct.c_char_p
    L.erq_build_index.argtypes = [vp, i64, i32, ct.POINTER(BuildParams), vp, ct.POINTER(vp)]
    L.erq_free_index.argtypes = [vp]
    L.erq_free_index.restype = None
    L.erq_index_info_get.argtypes = [vp, ct.POINTER(IndexInfo)]
    L.erq_index_status.argtypes = [vp, vp]
    L.erq_rotate.argtypes = [vp, i64, i32, vp, vp, i32, vp]
    L.erq_encode.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp, vp]
    L.erq_search.argtypes = [vp, vp, i64, ct.POINTER(SearchParams), vp, vp, vp]
    L.erq_search_host.argtypes = [vp, vp, i64, ct.POINTER(SearchParams), vp, vp, vp]
    L.erq_estimate.argtypes = [vp, vp, i64, i32, vp, vp, vp]
    L.erq_search_backward.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
    L.erq_estimate_metric.argtypes = [vp, vp, i64, i32, vp, i32, vp, vp]
    L.erq_search_backward_metric.argtypes = [vp, vp, i64, i32, vp, vp, i32, vp, vp]
    L.erq_index_export.argtypes = [vp, i32, vp, i64]
    L.erq_index_save.argtypes = [vp, ct.c_char_p]
    L.erq_index_load.argtypes = [ct.c_char_p, vp, ct.POINTER(vp)]
    L.erq_search_timing.argtypes = [vp, ct.POINTER(ct.c_float), i32]
    L.erq_search_timing_total.argtypes = [vp, ct.POINTER(ct.c_float), i32, ct.POINTER(ct.c_int64)]
    L.erq_autotune.argtypes = [vp, vp, i64, ct.POINTER(SearchParams), i32, vp, ct.POINTER(i32)]
    L.erq_set_scan_config.argtypes = [vp, i32, i32]
    L.erq_scan_config.argtypes = [vp, ct.POINTER(i32), i32]
    L.erq_kernel_launches.argtypes = []
    L.erq_kernel_launches.restype = ct.c_uint64
    L.erq_search_stats.argtypes = [vp, ct.POINTER(ct.c_int64), i32]
    L.erq_search_backward_noalloc.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
    L.erq_merge_topk.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, vp]
    L.erq_rerank_ids.argtypes = [vp, vp, i64, i32, vp, i32, i32, vp, vp, vp]
    L.erq_set_wait_limit.argtypes = [vp, ct.c_uint64, i64]
    L.erq_search_two_stage.argtypes = [vp, vp, i64, ct.POINTER(SearchParams), ct.c_float, vp, vp, vp, vp]
    for name in ("erq_build_index", "erq_index_info_get", "erq_index_status", "erq_rotate", "erq_encode",
                 "erq_search", "erq_search_host", "erq_estimate", "erq_search_backward", "erq_index_export",
                 "erq_index_save", "erq_index_load", "erq_search_timing",
                 "erq_search_stats", "erq_search_backward_noalloc", "erq_search_timing_total", "erq_autotune",
                 "erq_set_scan_config", "erq_scan_config"):
        getattr(L, name).restype = ct.c_int
    _lib = L
    return L


def _check(code):
    if code != ERQ_OK:
        raise ErqError(code, lib().erq_last_error().decode())


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ct.c_void_p(0 if t is None else t.data_ptr())


def _dev(t, dtype, name, ndim=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims")
    return t.contiguous()


def _check_out(out, like, name="out"):
    """A caller-supplied output buffer that the library writes through its raw
    pointer: a tensor of ``like``'s dtype and shape, contiguous, on the same
    CUDA device (anything else would be written out of bounds or in the wrong
    layout)."""
    if not isinstance(out, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if out.dtype != like.dtype:
        raise TypeError(f"{name} must be {like.dtype}, got {out.dtype}")
    if tuple(out.shape) != tuple(like.shape):
        raise ValueError(f"{name} must have shape {tuple(like.shape)}, got {tuple(out.shape)}")
    if not out.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not out.is_cuda or out.device != like.device:
        raise ValueError(f"{name} must be on {like.device}, got {out.device}")
    return out


def merge_topk(cand_ids, values, k, metric="l2"):
    """erq_merge_topk: per row, the k best (value, id) pairs of the candidate
    lists (device [nq, m] int64 ids, -1 = empty, and float32 values), ascending
    for "l2", descending for "ip"; returns (ids [nq, k], values [nq, k])."""
    cand_ids = _dev(cand_ids, torch.int64, "cand_ids", 2)
    values = _dev(values, torch.float32, "values", 2)
    if tuple(values.shape) != tuple(cand_ids.shape):
        raise ValueError("cand_ids and values must have the same shape")
    nq, m = cand_ids.shape
    ids = torch.empty((nq, k), dtype=torch.int64, device=cand_ids.device)
    vals = torch.empty((nq, k), dtype=torch.float32, device=cand_ids.device)
    _check(lib().erq_merge_topk(_ptr(cand_ids), _ptr(values), nq, m, int(k), METRIC[metric], _ptr(ids), _ptr(vals),
                                _stream()))
    return ids, vals


def kernel_launches() -> int:
    return int(lib().erq_kernel_launches())


def version() -> str:
    return lib().erq_version().decode()


def rotate(X, P, accurate=False, out=None):
    """out = X P (rows become P^T x); FP64 accumulation when accurate."""
    X = _dev(X, torch.float32, "X", 2)
    P = _dev(P, torch.float32, "P", 2)
    out = torch.empty_like(X) if out is None else out
    _check(lib().erq_rotate(_ptr(X), X.shape[0], X.shape[1], _ptr(P), _ptr(out), int(bool(accurate)), _stream()))
    return out


def encode(R, B, with_stats=False):
    """Algorithm 1 on each row of R (rotated residuals) -> (codes, f_add, f_res[, stats]);
    codes are uint8 for B <= 8 and 16-bit (int16, values < 2^B) for B = 9, 10."""
    R = _dev(R, torch.float32, "R", 2)
    n, d = R.shape
    codes = torch.empty((n, d), dtype=torch.int16 if int(B) > 8 else torch.uint8, device=R.device)
    f_add = torch.empty(n, dtype=torch.float32, device=R.device)
    f_res = torch.empty(n, dtype=torch.float32, device=R.device)
    stats = torch.empty((n, 2), dtype=torch.float64, device=R.device) if with_stats else None
    _check(lib().erq_encode(_ptr(R), n, d, int(B), _ptr(codes), _ptr(f_add), _ptr(f_res), _ptr(stats), _stream()))
    return (codes, f_add, f_res, stats) if with_stats else (codes, f_add, f_res)


class Index:
    """Owner of an erq_index (device memory freed with the object)."""

    def __init__(self, handle):
        self._h = ct.c_void_p(handle)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.erq_free_index(h)
            self._h = ct.c_void_p(0)

    def free(self):
        self.__del__()

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = IndexInfo()
        _check(lib().erq_index_info_get(self._h, ct.byref(inf)))
        return {f: getattr(inf, f) for f, _ in IndexInfo._fields_}

    def status(self):
        _check(lib().erq_index_status(self._h, _stream()))

    def search(self, Q, k, *, rerank_k=0, nprobe=1, precision="fp32", probe=None, nprobe_per_query=None,
               return_candidates=False, timing=False, simt_gemm=False, async_mode=False, metric="l2"):
        """erq_search.  metric "l2": squared distances, ascending; "ip": inner
        products, descending."""
        Q = _dev(Q, torch.float32, "Q", 2)
        nq = Q.shape[0]
        sp = SearchParams()
        sp.k, sp.rerank_k, sp.nprobe, sp.precision = int(k), int(rerank_k), int(nprobe), PREC[precision]
        sp.metric = METRIC[metric]
        sp.flags = (1 if timing else 0) | (2 if simt_gemm else 0) | (4 if async_mode else 0)
        keep = []
        if nprobe_per_query is not None:
            nprobe_per_query = _dev(nprobe_per_query, torch.int32, "nprobe_per_query", 1)
            keep.append(nprobe_per_query)
            sp.nprobe_per_query = nprobe_per_query.data_ptr()
        if probe is not None:
            probe = _dev(probe, torch.int32, "probe", 2)
            keep.append(probe)
            sp.probe = probe.data_ptr()
            sp.probe_stride = probe.shape[1]
        kc = max(int(k), int(rerank_k))
        cand_ids = cand_est = None
        if return_candidates:
            cand_ids = torch.empty((nq, kc), dtype=torch.int64, device=Q.device)
            cand_est = torch.empty((nq, kc), dtype=torch.float32, device=Q.device)
            sp.cand_ids, sp.cand_est = cand_ids.data_ptr(), cand_est.data_ptr()
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        _check(lib().erq_search(self._h, _ptr(Q), nq, ct.byref(sp), _ptr(ids), _ptr(dists), _stream()))
        if return_candidates:
            return ids, dists, cand_ids, cand_est
        return ids, dists

    def search_two_stage(self, Q, k, *, rerank_k=0, nprobe=1, eps0=1.9, probe=None, nprobe_per_query=None,
                         return_candidates=False, return_stats=False):
        """erq_search_two_stage (Section 4.2, metric l2): MSB-plane estimates
        with Lemma 2.1's bound (eps0) prune the probed rows, Eq. 4.2 completes
        the survivors.  return_stats adds (probed rows, survivors)."""
        Q = _dev(Q, torch.float32, "Q", 2)
        nq = Q.shape[0]
        sp = SearchParams()
        sp.k, sp.rerank_k, sp.nprobe, sp.precision = int(k), int(rerank_k), int(nprobe), PREC["fp32"]
        keep = []
        if nprobe_per_query is not None:
            nprobe_per_query = _dev(nprobe_per_query, torch.int32, "nprobe_per_query", 1)
            keep.append(nprobe_per_query)
            sp.nprobe_per_query = nprobe_per_query.data_ptr()
        if probe is not None:
            probe = _dev(probe, torch.int32, "probe", 2)
            keep.append(probe)
            sp.probe = probe.data_ptr()
            sp.probe_stride = probe.shape[1]
        kc = max(int(k), int(rerank_k))
        cand_ids = cand_est = None
        if return_candidates:
            cand_ids = torch.empty((nq, kc), dtype=torch.int64, device=Q.device)
            cand_est = torch.empty((nq, kc), dtype=torch.float32, device=Q.device)
            sp.cand_ids, sp.cand_est = cand_ids.data_ptr(), cand_est.data_ptr()
        ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        st = (ct.c_int64 * 2)()
        _check(lib().erq_search_two_stage(self._h, _ptr(Q), nq, ct.byref(sp), ct.c_float(eps0), _ptr(ids),
                                          _ptr(dists), st if return_stats else None, _stream()))
        out = (ids, dists) + ((cand_ids, cand_est) if return_candidates else ())
        if return_stats:
            out = out + ((int(st[0]), int(st[1])),)
        return out

    def timing(self):
        """Per-phase device ms of the last timed search: rotate, probe, plan, scan, merge, rerank."""
        ms = (ct.c_float * 6)()
        _check(lib().erq_search_timing(self._h, ms, 6))
        return dict(zip(("rotate", "probe", "plan", "scan", "merge", "rerank"), list(ms)))

    def autotune(self, Q, k, *, rerank_k=0, nprobe=1, precision="fp16", nprobe_per_query=None, reps=3, metric="l2"):
        """Time every supported scan work-item shape on this query batch and keep
        the fastest for later searches of this size; returns (queries per item,
        rows per item)."""
        Q = _dev(Q, torch.float32, "Q", 2)
        sp = SearchParams()
        sp.k, sp.rerank_k, sp.nprobe, sp.precision = int(k), int(rerank_k), int(nprobe), PREC[precision]
        sp.metric = METRIC[metric]
        keep = None
        if nprobe_per_query is not None:
            keep = _dev(nprobe_per_query, torch.int32, "nprobe_per_query", 1)
            sp.nprobe_per_query = keep.data_ptr()
        best = (ct.c_int32 * 2)()
        _check(lib().erq_autotune(self._h, _ptr(Q), Q.shape[0], ct.byref(sp), int(reps), _stream(), best))
        return int(best[0]), int(best[1])

    def set_scan_config(self, queries_per_item=0, rows_per_item=0):
        _check(lib().erq_set_scan_config(self._h, int(queries_per_item), int(rows_per_item)))

    def scan_config(self):
        out = (ct.c_int32 * 2)()
        _check(lib().erq_scan_config(self._h, out, 2))
        return int(out[0]), int(out[1])

    def timing_total(self):
        """Per-phase device ms summed over the timed searches since the previous
        call, and how many searches that covers."""
        ms = (ct.c_float * 6)()
        cnt = ct.c_int64()
        _check(lib().erq_search_timing_total(self._h, ms, 6, ct.byref(cnt)))
        return dict(zip(("rotate", "probe", "plan", "scan", "merge", "rerank"), list(ms))), cnt.value

    def stats(self):
        """Work of the last search: pairs, distinct rows, items, lists, tensor-core
        row blocks and row blocks x padded query count (the last two 0 for FP32)."""
        out = (ct.c_int64 * 6)()
        _check(lib().erq_search_stats(self._h, out, 6))
        return dict(zip(("pairs", "rows", "items", "lists", "blocks", "slot_blocks"), list(out)))

    def search_host(self, Q_host, k, *, rerank_k=0, nprobe=1, precision="fp32", async_mode=False,
                    nprobe_per_query=None, metric="l2"):
        """Search from host memory (pinned for asynchronous copies); returns host tensors.
        ``nprobe_per_query`` (optional) is a device int32 tensor [nq]."""
        if Q_host.is_cuda or Q_host.dtype != torch.float32:
            raise TypeError("Q_host must be a CPU float32 tensor")
        Q_host = Q_host.contiguous()
        nq = Q_host.shape[0]
        sp = SearchParams()
        sp.k, sp.rerank_k, sp.nprobe, sp.precision = int(k), int(rerank_k), int(nprobe), PREC[precision]
        sp.metric = METRIC[metric]
        sp.flags = 4 if async_mode else 0
        if nprobe_per_query is not None:
            nprobe_per_query = _dev(nprobe_per_query, torch.int32, "nprobe_per_query", 1)
            sp.nprobe_per_query = nprobe_per_query.data_ptr()
        pin = Q_host.is_pinned()
        ids = torch.empty((nq, k), dtype=torch.int64, pin_memory=pin)
        dists = torch.empty((nq, k), dtype=torch.float32, pin_memory=pin)
        _check(lib().erq_search_host(self._h, _ptr(Q_host), nq, ct.byref(sp), _ptr(ids), _ptr(dists), _stream()))
        return ids, dists

    def estimate(self, Q, ids, metric="l2"):
        """Estimated squared distances ("l2") or inner products ("ip") of Q[i] to ids[i, :]."""
        Q = _dev(Q, torch.float32, "Q", 2)
        ids = _dev(ids, torch.int64, "ids", 2)
        est = torch.empty(ids.shape, dtype=torch.float32, device=Q.device)
        _check(lib().erq_estimate_metric(self._h, _ptr(Q), Q.shape[0], ids.shape[1], _ptr(ids), METRIC[metric],
                                         _ptr(est), _stream()))
        return est

    def search_backward(self, Q, ids, grad_scores, metric="l2"):
        Q = _dev(Q, torch.float32, "Q", 2)
        ids = _dev(ids, torch.int64, "ids", 2)
        g = _dev(grad_scores, torch.float32, "grad_scores", 2)
        out = torch.empty_like(Q)
        _check(lib().erq_search_backward_metric(self._h, _ptr(Q), Q.shape[0], ids.shape[1], _ptr(ids), _ptr(g),
                                                METRIC[metric], _ptr(out), _stream()))
        return out

    def search_backward_noalloc(self, Q, ids, grad_scores, out=None):
        """erq_search_backward without device allocation inside the call (its
        intermediates live in the library's fixed scratch array); ``out`` may be
        a preallocated contiguous [nq, D] float32 tensor on Q's device (checked:
        TypeError / ValueError otherwise)."""
        Q = _dev(Q, torch.float32, "Q", 2)
        ids = _dev(ids, torch.int64, "ids", 2)
        g = _dev(grad_scores, torch.float32, "grad_scores", 2)
        out = torch.empty_like(Q) if out is None else _check_out(out, Q)
        _check(lib().erq_search_backward_noalloc(self._h, _ptr(Q), Q.shape[0], ids.shape[1], _ptr(ids), _ptr(g),
                                                 _ptr(out), _stream()))
        return out

    def rerank_ids(self, Q, ids, k, metric="l2"):
        """erq_rerank_ids: exact re-rank of the given ids (device [nq, nc] int64,
        ids this index does not hold are skipped); returns (ids, distances or
        inner products) [nq, k]."""
        Q = _dev(Q, torch.float32, "Q", 2)
        ids = _dev(ids, torch.int64, "ids", 2)
        nq, nc = ids.shape
        out_i = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
        out_d = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        _check(lib().erq_rerank_ids(self._h, _ptr(Q), nq, nc, _ptr(ids), int(k), METRIC[metric], _ptr(out_i),
                                    _ptr(out_d), _stream()))
        return out_i, out_d

    def set_wait_limit(self, ns, stall_stage=-1):
        """Limit of the scan's bounded device-side waits in ns (0 = default 2 s);
        stall_stage >= 0 makes later scans wait at that stage on a barrier that
        nothing arrives on (a test of the ERQ_ETIMEOUT path)."""
        _check(lib().erq_set_wait_limit(self._h, int(ns), int(stall_stage)))

    def export(self, field):
        inf = self.info()
        N, D, nl = inf["N"], inf["D"], inf["nlist"]
        shapes = {"centroids": ((nl, D), torch.float32), "rot_centroids": ((nl, D), torch.float32),
                  "list_offsets": ((nl + 1,), torch.int64), "list_ids": ((N,), torch.int64),
                  "codes": ((N, D), torch.int16 if inf["B"] > 8 else torch.uint8), "f_add": ((N,), torch.float32),
                  "f_res": ((N,), torch.float32),
                  "P": ((D, D), torch.float32), "raw": ((N, D), torch.float32)}
        if field == "packed_codes":      # clusters padded to 32-row tiles, B bits per coordinate
            off = self.export("list_offsets")
            Np = int(((off[1:] - off[:-1] + 31) // 32 * 32).sum())
            shapes[field] = ((Np * D * inf["B"] // 8,), torch.uint8)
        shape, dt = shapes[field]
        out = torch.empty(shape, dtype=dt)
        torch.cuda.current_stream().synchronize()
        _check(lib().erq_index_export(self._h, FIELDS[field], _ptr(out), out.numel() * out.element_size()))
        return out

    def save(self, path):
        torch.cuda.current_stream().synchronize()
        _check(lib().erq_index_save(self._h, str(path).encode()))

    @staticmethod
    def load(path):
        h = ct.c_void_p()
        _check(lib().erq_index_load(str(path).encode(), _stream(), ct.byref(h)))
        return Index(h.value)


def build_index(X, P, B, nlist=1, *, assign=None, keep_raw=True, kmeans_iters=10, kmeans_sample=0, seed=0,
                centroids=None, normalize=False):
    """Build an IVF + extended-RaBitQ index from device rows X [N, D].
    ``centroids`` (device [nlist, D], with ``assign``): use these instead of the
    means of the rows (an index over one shard of a larger index's lists).
    ``normalize``: scale the rows to unit length first (searches with
    metric "cos")."""
    X = _dev(X, torch.float32, "X", 2)
    P = _dev(P, torch.float32, "P", 2)
    bp = BuildParams()
    bp.B, bp.nlist, bp.P = int(B), int(nlist), P.data_ptr()
    bp.normalize = 1 if normalize else 0
    if assign is not None:
        assign = _dev(assign, torch.int32, "assign", 1)
        bp.assign = assign.data_ptr()
    if centroids is not None:
        centroids = _dev(centroids, torch.float32, "centroids", 2)
        if tuple(centroids.shape) != (int(nlist), X.shape[1]):
            raise ValueError(f"centroids must have shape ({int(nlist)}, {X.shape[1]})")
        bp.centroids = centroids.data_ptr()
    bp.kmeans_iters, bp.kmeans_sample, bp.seed, bp.keep_raw = int(kmeans_iters), int(kmeans_sample), int(seed), \
        int(bool(keep_raw))
    h = ct.c_void_p()
    _check(lib().erq_build_index(_ptr(X), X.shape[0], X.shape[1], ct.byref(bp), _stream(), ct.byref(h)))
    return Index(h.value)
