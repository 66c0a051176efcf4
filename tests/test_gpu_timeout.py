"""Failure detection on the GPU without a GPU fault: every wait of the
tensor-core scan is bounded.  With a test stall set (erq_set_wait_limit with
stall_stage >= 0) the first MMA issuer of every CTA waits, in the middle of
the pipeline, on a barrier that nothing arrives on; after the limit (20 ms)
the scan must stop, drain its copies and MMAs, free its tensor memory and
report ERQ_ETIMEOUT through the index's status word, and the same index must
then search correctly again with the stall off and the default limit."""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_common import erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kp,precision", [(20, "fp16"), (100, "fp16"), (24, "fp8")])
def test_scan_wait_limit_times_out_and_index_recovers(erq, kp, precision):
    X, lab = S.mixture(20000, 128, 16, 6100, scale="aniso")
    assign = S.kmeans_assign(X, 32, 3, 6101)
    P = S.random_orthogonal(128, 6102)
    B = 4 if precision == "fp8" else 5
    gx = erq.build_index(to_dev(X), to_dev(P), B, 32, assign=to_dev(assign))
    Q = to_dev(S.mixture(600, 128, 16, 6103, comp_seed=6100, scale="aniso")[0])
    kw = dict(rerank_k=kp, nprobe=6, precision=precision, return_candidates=True)
    ref = gx.search(Q, 10, **kw)
    torch.cuda.synchronize()
    gx.status()
    gx.set_wait_limit(20_000_000, stall_stage=1)   # a wait on a barrier nothing arrives on, limit 20 ms
    gx.search(Q, 10, **kw)
    with pytest.raises(erq.ErqError) as ei:
        gx.status()
    assert ei.value.code == erq.ERQ_ETIMEOUT
    gx.status()                                # the status word was cleared by the read
    gx.set_wait_limit(0)                       # no stall, the default limit
    for _ in range(2):                         # tensor memory was freed: later scans allocate it again
        got = gx.search(Q, 10, **kw)
        torch.cuda.synchronize()
        gx.status()
        for a, b in zip(ref, got):
            assert torch.equal(a, b)
