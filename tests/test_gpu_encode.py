"""GPU parity: rotation and encoder (Algorithm 1) against the FP64 oracle.

Codes, both stored factors and the FP64 optimum statistics must match
bit-exactly when both sides receive the same FP32 rotated residuals."""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from gpu_common import erq, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _check_encode(erq, R, B):
    codes_o, st_o = oracle.quantize(R, B)
    fa_o, fr_o = oracle.stored_factors(st_o)
    codes, fa, fr, st = erq.encode(to_dev(R), B, with_stats=True)
    torch.cuda.synchronize()
    codes, fa, fr, st = codes.cpu().numpy(), fa.cpu().numpy(), fr.cpu().numpy(), st.cpu().numpy()
    bad = np.nonzero((codes != codes_o).any(1))[0]
    assert len(bad) == 0, f"B={B}: {len(bad)} rows with different codes, first {bad[:5]}"
    np.testing.assert_array_equal(st[:, 0], st_o[:, 0])          # <ybar,|o'|> at the optimum, bit-exact
    np.testing.assert_array_equal(st[:, 1], st_o[:, 1])          # ||ybar||^2
    np.testing.assert_array_equal(fa.view(np.uint32), fa_o.view(np.uint32))
    np.testing.assert_array_equal(fr.view(np.uint32), fr_o.view(np.uint32))


@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("kind", ["gauss", "ties", "sparse", "wide"])
def test_encode_bit_exact_d128(erq, B, kind):
    R = S.random_rotated_residuals(300, 128, 1000 + B, kind=kind)
    _check_encode(erq, R, B)


@pytest.mark.parametrize("D,B,n", [(64, 5, 400), (960, 3, 200), (960, 5, 200), (960, 7, 60), (1536, 7, 40),
                                   (768, 5, 150), (1024, 4, 150), (4096, 2, 20), (960, 9, 20),
                                   (960, 10, 12), (4096, 10, 3)])
def test_encode_bit_exact_paper_shapes(erq, D, B, n):
    R = S.random_rotated_residuals(n, D, 2000 + D + B)
    _check_encode(erq, R, B)


@pytest.mark.parametrize("B", [4, 6, 8, 10])
def test_encode_bit_exact_openai3072(erq, B):
    """The Table 4 shape (D = 3072), with a few very small coordinates planted
    in half of the rows: their events make FP64 additions of the running
    <y, o'> round, which the encoder must reproduce in order."""
    R = S.random_rotated_residuals(10, 3072, 2600 + B)
    R[::2, 7:10] *= np.float32(3e-5)
    R[1::4, 100] = np.float32(1e-7)
    _check_encode(erq, R, B)


def test_encode_degenerate_rows(erq):
    """Zero vector (reading R8), single non-zero, all-equal magnitudes (maximal
    event ties), magnitudes spanning 2^100 both ways."""
    D = 64
    rows = np.zeros((6, D), np.float32)
    rows[1, 5] = -3.0
    rows[2] = np.where(np.arange(D) % 2 == 0, 1.0, -1.0)
    rows[3, :] = 1.0
    rows[4, 0], rows[4, 1:] = 2.0 ** -101, 0.5
    rows[5, 0], rows[5, 1:] = 1e30, 1.0
    for B in (1, 2, 4, 8, 9, 10):
        _check_encode(erq, rows, B)


def test_encode_rejects_extreme_range(erq):
    """A non-zero coordinate below 2^-118 of the row's largest is outside the
    encoder's documented domain and is reported, not silently mis-ordered."""
    rows = np.full((1, 64), 1.0, np.float32)
    rows[0, 3] = 1e-40
    with pytest.raises(erq.ErqError, match="2\\^-118"):
        erq.encode(to_dev(rows), 4)


def test_encode_empty_and_invalid(erq):
    codes, fa, fr = erq.encode(torch.zeros((0, 64), device="cuda"), 4)
    assert codes.shape == (0, 64)
    with pytest.raises(erq.ErqError):
        erq.encode(torch.zeros((2, 65), device="cuda"), 4)
    with pytest.raises(erq.ErqError):
        erq.encode(torch.zeros((2, 64), device="cuda"), 11)


@pytest.mark.parametrize("D", [64, 960])
def test_rotate_fp64_bit_exact(erq, D):
    X, _ = S.mixture(333, D, 4, 3000 + D)
    P = S.random_orthogonal(D, 3001)
    got = erq.rotate(to_dev(X), to_dev(P), accurate=True).cpu().numpy()
    ref = oracle.rotate(X, P)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_rotate_fp32_close(erq):
    D = 256
    X, _ = S.mixture(1000, D, 4, 3100)
    P = S.random_orthogonal(D, 3101)
    got = erq.rotate(to_dev(X), to_dev(P), accurate=False).cpu().numpy().astype(np.float64)
    ref = X.astype(np.float64) @ P.astype(np.float64)
    err = np.abs(got - ref).max(1) / np.linalg.norm(ref, axis=1)
    assert err.max() < 1e-6


@pytest.mark.parametrize("nlist,N", [(1, 2000), (8, 3001), (37, 5000)])
def test_build_index_bit_exact(erq, nlist, N):
    """Centroids (FP64 means), lists, codes and factors of the whole index equal
    the oracle's index built from the same rows, P and assignment."""
    D, B = 128, 4
    X, lab = S.mixture(N, D, max(nlist, 2), 4000 + nlist)
    assign = (lab % nlist).astype(np.int32) if nlist > 1 else np.zeros(N, np.int32)
    if nlist == 37:
        assign[assign == 5] = 6          # an empty cluster
    P = S.random_orthogonal(D, 4001)
    ix = erq.build_index(to_dev(X), to_dev(P), B, nlist, assign=to_dev(assign))
    ref = oracle.build_index(X, P, assign, nlist, B)
    np.testing.assert_array_equal(ix.export("centroids").numpy().view(np.uint32), ref["C"].view(np.uint32))
    np.testing.assert_array_equal(ix.export("rot_centroids").numpy().view(np.uint32), ref["Cp"].view(np.uint32))
    np.testing.assert_array_equal(ix.export("list_offsets").numpy(), ref["list_off"])
    np.testing.assert_array_equal(ix.export("list_ids").numpy(), ref["list_ids"])
    np.testing.assert_array_equal(ix.export("codes").numpy(), ref["codes"])
    fa_o, fr_o = oracle.stored_factors(ref["stats"])
    np.testing.assert_array_equal(ix.export("f_add").numpy().view(np.uint32), fa_o.view(np.uint32))
    np.testing.assert_array_equal(ix.export("f_res").numpy().view(np.uint32), fr_o.view(np.uint32))
    info = ix.info()
    assert info["N"] == N and info["nlist"] == nlist and info["max_list"] == np.diff(ref["list_off"]).max()


def test_build_rejects_bad_assignment(erq):
    D = 64
    X, _ = S.mixture(500, D, 2, 4100)
    P = S.random_orthogonal(D, 4101)
    assign = np.zeros(500, np.int32)
    assign[7] = 9
    with pytest.raises(erq.ErqError):
        erq.build_index(to_dev(X), to_dev(P), 4, 4, assign=to_dev(assign))


def test_save_load_roundtrip(erq, tmp_path):
    D = 64
    X, lab = S.mixture(800, D, 3, 4200)
    P = S.random_orthogonal(D, 4201)
    ix = erq.build_index(to_dev(X), to_dev(P), 5, 3, assign=to_dev(lab))
    path = tmp_path / "ix.bin"
    ix.save(path)
    ix2 = erq.Index.load(path)
    for f in ("codes", "f_add", "f_res", "centroids", "list_ids", "raw"):
        np.testing.assert_array_equal(ix.export(f).numpy(), ix2.export(f).numpy())
    Q = to_dev(S.mixture(5, D, 3, 4202, comp_seed=4200)[0])
    a = ix.search(Q, 5, rerank_k=20, nprobe=2)
    b = ix2.search(Q, 5, rerank_k=20, nprobe=2)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
