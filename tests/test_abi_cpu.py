"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point declared in include/erq.h, and rejects bad arguments on the
host before any CUDA work (no GPU needed)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2409_09913_gb300 import build, erq
    build.build()
    return erq.lib()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "erq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(erq_[a-z_]+)\s*\(", src)))


def test_header_functions_are_exported(L):
    names = _header_functions()
    assert len(names) >= 15
    from paper_2409_09913_gb300 import erq
    assert sorted(erq.EXPORTS) == names
    for n in names:
        assert hasattr(L, n), n


def test_version_and_last_error(L):
    from paper_2409_09913_gb300 import erq
    assert "sm_103a" in erq.version()
    assert isinstance(L.erq_last_error(), bytes)


def _vp(v=0):
    return ct.c_void_p(v)


def test_host_validation_rejects_bad_shapes(L):
    from paper_2409_09913_gb300 import erq
    # D not a multiple of 64
    assert L.erq_rotate(_vp(8), 4, 63, _vp(8), _vp(8), 0, _vp()) == erq.ERQ_EINVAL
    assert b"multiple of 64" in L.erq_last_error()
    # B out of range
    assert L.erq_encode(_vp(8), 4, 64, 11, _vp(8), _vp(8), _vp(8), _vp(), _vp()) == erq.ERQ_EINVAL
    assert L.erq_encode(_vp(8), 4, 64, 0, _vp(8), _vp(8), _vp(8), _vp(), _vp()) == erq.ERQ_EINVAL
    # null pointers
    assert L.erq_encode(_vp(0), 4, 64, 4, _vp(8), _vp(8), _vp(8), _vp(), _vp()) == erq.ERQ_EINVAL
    # n == 0 is a no-op
    assert L.erq_encode(_vp(0), 0, 64, 4, _vp(0), _vp(0), _vp(0), _vp(), _vp()) == erq.ERQ_OK


def test_host_validation_build_params(L):
    from paper_2409_09913_gb300 import erq
    out = ct.c_void_p()
    bp = erq.BuildParams()
    bp.B, bp.nlist, bp.P = 4, 1, 0
    assert L.erq_build_index(_vp(8), 100, 64, ct.byref(bp), _vp(), ct.byref(out)) == erq.ERQ_EINVAL
    bp.P, bp.B = 8, 10
    assert L.erq_build_index(_vp(8), 100, 64, ct.byref(bp), _vp(), ct.byref(out)) == erq.ERQ_EINVAL
    bp.B, bp.nlist = 4, 101
    assert L.erq_build_index(_vp(8), 100, 64, ct.byref(bp), _vp(), ct.byref(out)) == erq.ERQ_EINVAL
    bp.nlist = 4
    assert L.erq_build_index(_vp(8), 100, 100, ct.byref(bp), _vp(), ct.byref(out)) == erq.ERQ_EINVAL
    assert L.erq_build_index(_vp(8), 0, 64, ct.byref(bp), _vp(), ct.byref(out)) == erq.ERQ_EINVAL
    assert out.value is None


def test_search_validation_needs_index(L):
    from paper_2409_09913_gb300 import erq
    sp = erq.SearchParams()
    sp.k = 10
    assert L.erq_search(_vp(0), _vp(8), 1, ct.byref(sp), _vp(8), _vp(8), _vp()) == erq.ERQ_EINVAL


def test_load_rejects_missing_and_corrupt_files(L, tmp_path):
    from paper_2409_09913_gb300 import erq
    out = ct.c_void_p()
    assert L.erq_index_load(str(tmp_path / "nope.bin").encode(), _vp(), ct.byref(out)) == erq.ERQ_EIO
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTANIDX" + b"\0" * 64)
    assert L.erq_index_load(str(bad).encode(), _vp(), ct.byref(out)) == erq.ERQ_EIO
    assert b"magic" in L.erq_last_error()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2409_09913_gb300 import erq
    monkeypatch.setattr(erq, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        erq.lib(str(tmp_path / "missing.so"))


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the header's size and field offsets."""
    import shutil
    import subprocess
    from paper_2409_09913_gb300 import erq
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "erq.h"\n'
                   'int main(void) {\n'
                   '  printf("%zu %zu %zu %zu\\n", sizeof(erq_search_params), offsetof(erq_search_params, metric),\n'
                   '         offsetof(erq_search_params, cand_est), sizeof(erq_build_params));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    size, off_metric, off_est, bsize = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                               text=True).stdout.split())
    assert ct.sizeof(erq.SearchParams) == size
    assert erq.SearchParams.metric.offset == off_metric
    assert erq.SearchParams.cand_est.offset == off_est
    assert ct.sizeof(erq.BuildParams) == bsize


def test_metric_entry_points_validate_on_host(L):
    """The metric variants reject bad arguments before any device work."""
    from paper_2409_09913_gb300 import erq
    assert L.erq_estimate_metric(_vp(0), _vp(8), 1, 1, _vp(8), 1, _vp(8), _vp()) == erq.ERQ_EINVAL
    assert L.erq_search_backward_metric(_vp(0), _vp(8), 1, 1, _vp(8), _vp(8), 1, _vp(8), _vp()) == erq.ERQ_EINVAL
    assert b"bad arguments" in L.erq_last_error()


def test_noalloc_output_buffer_is_checked_before_the_call():
    """The allocation-free backward writes nq * D floats through the raw
    pointer of a caller-supplied ``out``; the binding rejects a buffer of the
    wrong dtype, shape, layout or device before any library call."""
    import torch
    from paper_2409_09913_gb300 import erq
    like = torch.zeros((3, 64))
    with pytest.raises(ValueError, match="shape"):
        erq._check_out(torch.zeros((3, 63)), like)
    with pytest.raises(ValueError, match="shape"):
        erq._check_out(torch.zeros((2, 64)), like)
    with pytest.raises(TypeError, match="float32"):
        erq._check_out(torch.zeros((3, 64), dtype=torch.float64), like)
    with pytest.raises(ValueError, match="contiguous"):
        erq._check_out(torch.zeros((64, 3)).t(), like)
    with pytest.raises(ValueError, match="must be on"):
        erq._check_out(torch.zeros((3, 64)), like)          # not a CUDA tensor
    with pytest.raises(TypeError):
        erq._check_out(None, like)
