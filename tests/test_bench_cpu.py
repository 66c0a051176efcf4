"""Host logic of the benchmark that needs no GPU: the DRAM-traffic lookup that
fills the roofline's "traffic" field from the committed ncu capture."""
import os
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
sys.path.insert(0, ROOT)


@pytest.fixture()
def bench_mod(tmp_path, monkeypatch):
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "scan_tc_traffic_w.txt").write_text(
        "# a capture\n"
        "workload: w\nnprobe: 16\nkernel_source_sha256: abc\n"
        "record: queries_per_item=64 rows_per_item=4096,8192 work_items=1000 dram_bytes_per_launch=5e8\n"
        "record: queries_per_item=64 rows_per_item=2048 work_items=1100 dram_bytes_per_launch=6e8\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "scan_source_sha", lambda: "abc")
    return bench


def test_traffic_matches_captured_shape(bench_mod):
    t = bench_mod.profiled_traffic
    assert t("w", 16, "fp16", (64, 4096), 999) == 5e8        # listed row limit wins
    assert t("w", 16, "fp16", (64, 8192), None) == 5e8
    assert t("w", 16, "fp16", (64, 2048), 1100) == 6e8
    assert t("w", 16, "fp16", (64, 512), 1004) == 5e8        # unlisted rows, item count within 0.5 %
    assert t("w", 16, "fp16", (64, 512), 1010) is None
    assert t("w", 16, "fp16", (32, 4096), 1000) is None      # other queries per item
    assert t("w", 32, "fp16", (64, 4096), 1000) is None      # other nprobe
    assert t("w", 16, "fp32", (64, 4096), 1000) is None      # the FP32 scan has no capture
    assert t("other", 16, "fp16", (64, 4096), 1000) is None  # no file


def test_traffic_dropped_when_kernel_source_changes(bench_mod, monkeypatch):
    monkeypatch.setattr(bench_mod, "scan_source_sha", lambda: "def")
    assert bench_mod.profiled_traffic("w", 16, "fp16", (64, 4096), 1000) is None



def test_oracle_sample_respects_row_cap():
    """The timed CPU sample takes queries in order while the rows of their
    probed clusters stay within --cpu-rows (at least one query), with the
    workload's per-query nprobe."""
    import argparse

    import numpy as np

    import bench
    import synthetic as S
    X, lab = S.mixture(4000, 64, 8, 11)
    Q, _ = S.mixture(6, 64, 8, 12, comp_seed=11)
    P = S.random_orthogonal(64, 13)
    cfg = {"nlist": 8}
    args = argparse.Namespace(metric="l2", B=3, cpu_rows=10 ** 9)
    ox, Qs, rows, npq = bench.oracle_sample(cfg, X, Q, P, lab, args, 2, 10, 16)
    assert len(Qs) == 6 and (npq == 2).all()
    args.cpu_rows = 1
    ox, Qs, rows, npq = bench.oracle_sample(cfg, X, Q, P, lab, args, 0, 10, 16, npr=np.array([3, 1, 1, 1, 1, 1]))
    assert len(Qs) == 1 and npq.tolist() == [3]
    assert len(np.unique(lab[rows])) == 3 and len(rows) == np.isin(lab, np.unique(lab[rows])).sum()
