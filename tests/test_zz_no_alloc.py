"""The allocation-free backward entry point.

erq_search_backward_noalloc serves callers that cannot allocate device memory
during the call (for example a host whose device memory comes from its own
pool).
It must give the same gradient as erq_search_backward, which allocates its
workspace, on consecutive calls that share the fixed scratch array, and it
must refuse requests larger than that array."""
import ctypes as ct

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _case(seed, N=3000, D=128, nq=17, nc=23):
    X, lab = S.mixture(N, D, 5, seed, scale="aniso")
    Q, _ = S.mixture(nq, D, 5, seed + 1, comp_seed=seed, scale="aniso")
    ids = np.stack([S.rng(seed + 2 + i).choice(N, nc, replace=False) for i in range(nq)]).astype(np.int64)
    ids[0, 1] = -1
    g = S.normal((nq, nc), seed + 99)
    return X, lab, Q, ids, g


def test_noalloc_backward_matches_allocating_entry_point():
    from paper_2409_09913_gb300 import build, erq
    build.build()
    L = erq.lib()
    dev = torch.device("cuda:0")
    X, lab, _, _, _ = _case(5100)
    P = S.random_orthogonal(128, 5101)
    ix = erq.build_index(torch.from_numpy(X).to(dev), torch.from_numpy(P).to(dev), 4, 5,
                         assign=torch.from_numpy(lab).to(dev))
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((5200, 5300)):          # two calls in a row share the scratch
        _, _, Q, ids, g = _case(seed, nq=17 + 6 * call, nc=23 - 5 * call)
        Qd = torch.from_numpy(Q).to(dev)
        idd = torch.from_numpy(ids).to(dev)
        gd = torch.from_numpy(g).to(dev)
        ref = ix.search_backward(Qd, idd, gd)
        out = torch.full_like(Qd, float("nan"))
        rc = L.erq_search_backward_noalloc(ix.handle, ct.c_void_p(Qd.data_ptr()), Qd.shape[0], idd.shape[1],
                                           ct.c_void_p(idd.data_ptr()), ct.c_void_p(gd.data_ptr()),
                                           ct.c_void_p(out.data_ptr()), stream)
        assert rc == erq.ERQ_OK, L.erq_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all()
        assert np.abs(a - b).max() <= 2e-5 * np.abs(b).max()


def test_noalloc_backward_size_limit_and_output_buffer():
    from paper_2409_09913_gb300 import erq
    dev = torch.device("cuda:0")
    X, lab, _, _, _ = _case(5400, N=1000, D=1024)
    P = S.random_orthogonal(1024, 5401)
    ix = erq.build_index(torch.from_numpy(X).to(dev), torch.from_numpy(P).to(dev), 3, 5,
                         assign=torch.from_numpy(lab).to(dev))
    # 8 nq D + 4 nq + 512 <= 16 MiB holds for nq = 2046 at D = 1024 and not for 2047
    nq = 2046
    Q = torch.from_numpy(S.normal((nq, 1024), 5402)).to(dev)
    ids = torch.from_numpy(S.rng(5403).integers(0, 1000, size=(nq, 2))).to(dev)
    g = torch.from_numpy(S.normal((nq, 2), 5404)).to(dev)
    out = torch.full_like(Q, float("nan"))
    got = ix.search_backward_noalloc(Q, ids, g, out=out)   # a preallocated output is written in place
    ref = ix.search_backward(Q, ids, g)
    torch.cuda.synchronize()
    assert got.data_ptr() == out.data_ptr()
    a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    assert np.isfinite(a).all() and np.abs(a - b).max() <= 2e-5 * np.abs(b).max()
    nq = 2047                                              # one query more than the scratch holds
    Q = torch.zeros((nq, 1024), device=dev)
    ids = torch.zeros((nq, 1), dtype=torch.int64, device=dev)
    g = torch.zeros((nq, 1), device=dev)
    with pytest.raises(erq.ErqError, match="scratch"):
        ix.search_backward_noalloc(Q, ids, g)
    with pytest.raises(ValueError, match="shape"):        # a wrong-shaped output is refused by the binding
        ix.search_backward_noalloc(Q[:5], ids[:5], g[:5], out=torch.empty((5, 512), device=dev))
