"""The checked build (-DERQ_CHECKS): every index a kernel derives from device
data (list and item slots, query-list entries, row ids of candidates) is
compared with its allocation; a failed check sets a status bit per site and
skips the access.  Searches over the precisions, k' classes and launch modes
must leave the status clean."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))

SCRIPT = textwrap.dedent("""
    import sys, numpy as np, torch
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    from paper_2409_09913_gb300 import build
    build.build(checked=True)
    from paper_2409_09913_gb300 import erq
    assert erq.lib()._name.endswith("liberq_checked.so"), erq.lib()._name
    import synthetic as S
    dev = torch.device("cuda", 0)
    for D, B in ((128, 4), (192, 5)):
        X, _ = S.mixture(20000, D, 16, 4200 + D, scale="aniso")
        assign = S.kmeans_assign(X, 48, 4, 4201)
        P = S.random_orthogonal(D, 4202)
        gx = erq.build_index(torch.from_numpy(X).to(dev), torch.from_numpy(P).to(dev), B, 48,
                             assign=torch.from_numpy(assign).to(dev))
        Q = torch.from_numpy(S.mixture(700, D, 16, 4203, comp_seed=4200 + D, scale="aniso")[0]).to(dev)
        npr = torch.from_numpy(np.random.default_rng(4204).integers(1, 13, 700).astype(np.int32)).to(dev)
        precs = ("fp32", "fp16", "fp8")
        for prec in precs:
            for kp in (20, 100):
                for am in (False, True):
                    gx.search(Q, 10, rerank_k=kp, nprobe=12, precision=prec, async_mode=am)
                    gx.search(Q, 10, rerank_k=kp, nprobe=12, precision=prec, async_mode=am, nprobe_per_query=npr)
            torch.cuda.synchronize()
        gx.status()          # raises with the failed sites, if any
    print("CHECKED-CLEAN")
""")


def test_checked_build_searches_clean():
    env = dict(os.environ, ERQ_CHECKED="1")
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED-CLEAN" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
