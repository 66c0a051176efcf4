"""Seeded synthetic inputs for the extended-RaBitQ search path.

This module is the only code shared by the CPU oracle (``oracle/``) and the
GPU path (``paper_2409_09913_gb300``).  It draws random numbers and nothing
else: it holds none of the method's arithmetic (no rotation applied, no
quantization, no distance estimation).  Random quantities that the method
itself draws -- the orthogonal matrix P (Section 2.2, Eq. "codebook rabitq";
Section 3.1, Eq. "equ:rotation") -- are produced here and handed to both sides
as inputs.

Workload shapes follow the paper's datasets (Table 1: million-scale embeddings
with D between 300 and 3072, IVF with 4,096 clusters per Section 5.1) as
Gaussian mixtures, because the real datasets are not available:

* ``mixture``: K components, centres ~ N(0, centre_std^2 I), per-component
  per-dimension standard deviations either 1 (isotropic) or ~ U(lo, hi)
  (anisotropic), component weights equal or Zipf(s); optional L2
  normalisation of every row (embedding-like data).
* queries are drawn from the same mixture with a different seed.

All generators use numpy's PCG64 so that a (seed, shape) pair names one input.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "mixture",
    "random_orthogonal",
    "zipf_weights",
    "random_rotated_residuals",
    "random_assign",
    "random_probe_lists",
    "uniform_ints",
    "normal",
    "kmeans_assign",
    "kmeans_assign_torch",
    "WORKLOADS",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def zipf_weights(n: int, s: float) -> np.ndarray:
    """Normalised Zipf(s) weights w_k proportional to 1/k^s, k = 1..n (FP64)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    w = 1.0 / k ** s
    return w / w.sum()


def mixture(n: int, d: int, n_comp: int, seed: int, *, centre_std: float = 2.0,
            scale: str = "unit", scale_lo: float = 0.5, scale_hi: float = 2.0,
            weights: np.ndarray | None = None, normalize: bool = False,
            comp_seed: int | None = None, exact_sizes: bool = False,
            chunk: int = 1 << 16):
    """Draw ``n`` rows of a ``d``-dimensional Gaussian mixture.

    The mixture itself (centres, scales) is drawn from ``comp_seed`` (defaults
    to ``seed``) so that base data and queries can share one mixture while
    using different sample seeds.  Returns ``(X float32 [n, d], labels int32)``.
    With ``exact_sizes`` the component sizes are round(n * w_k) (rest to the
    largest), otherwise labels are sampled i.i.d. from the weights.
    """
    cs = seed if comp_seed is None else comp_seed
    g_comp = rng(cs)
    centres = g_comp.normal(0.0, centre_std, size=(n_comp, d))
    if scale == "unit":
        scales = np.ones((n_comp, d))
    elif scale == "aniso":
        scales = g_comp.uniform(scale_lo, scale_hi, size=(n_comp, d))
    else:
        raise ValueError(scale)
    w = np.full(n_comp, 1.0 / n_comp) if weights is None else np.asarray(weights, np.float64)
    g = rng(seed)
    if exact_sizes:
        sizes = np.floor(w * n).astype(np.int64)
        sizes[0] += n - sizes.sum()
        labels = np.repeat(np.arange(n_comp, dtype=np.int32), sizes)
        g.shuffle(labels)
    else:
        labels = g.choice(n_comp, size=n, p=w).astype(np.int32)
    X = np.empty((n, d), dtype=np.float32)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        lab = labels[s0:s1]
        z = g.standard_normal(size=(s1 - s0, d))
        blk = centres[lab] + z * scales[lab]
        if normalize:
            blk /= np.linalg.norm(blk, axis=1, keepdims=True)
        X[s0:s1] = blk.astype(np.float32)
    return X, labels


def random_orthogonal(d: int, seed: int) -> np.ndarray:
    """A random orthogonal matrix, the method's only random draw.

    Gaussian d x d matrix, Householder QR in FP64, columns sign-fixed by the
    signs of diag(R) so that the draw is Haar-distributed, then stored as
    FP32.  Both the oracle and the GPU path treat the FP32 values as exact.
    """
    g = rng(seed)
    a = g.standard_normal(size=(d, d))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q.astype(np.float32))


def random_rotated_residuals(n: int, d: int, seed: int, *, kind: str = "gauss") -> np.ndarray:
    """FP32 rows standing in for rotated residuals r' (encoder inputs).

    ``gauss``: i.i.d. N(0,1); ``ties``: small integers (many exact event
    ties); ``sparse``: ~30% exact zeros; ``wide``: log-uniform magnitudes over
    20 binades with random signs.
    """
    g = rng(seed)
    if kind == "gauss":
        x = g.standard_normal(size=(n, d))
    elif kind == "ties":
        x = g.integers(-4, 5, size=(n, d)).astype(np.float64)
    elif kind == "sparse":
        x = g.standard_normal(size=(n, d)) * (g.random(size=(n, d)) > 0.3)
    elif kind == "wide":
        x = np.exp2(g.uniform(-20, 0, size=(n, d))) * np.where(g.random(size=(n, d)) < 0.5, -1.0, 1.0)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(x.astype(np.float32))


def random_assign(n: int, nlist: int, seed: int) -> np.ndarray:
    return rng(seed).integers(0, nlist, size=n).astype(np.int32)


def random_probe_lists(nq: int, nlist: int, nprobe: int, seed: int) -> np.ndarray:
    """``nq`` rows of ``nprobe`` distinct cluster ids drawn uniformly."""
    g = rng(seed)
    out = np.empty((nq, nprobe), dtype=np.int32)
    for i in range(nq):
        out[i] = g.choice(nlist, size=nprobe, replace=False)
    return out


def uniform_ints(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``n`` integers uniform on {lo..hi} inclusive."""
    return rng(seed).integers(lo, hi + 1, size=n).astype(np.int32)


def normal(shape, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(size=shape).astype(np.float32)


def kmeans_assign(X: np.ndarray, nlist: int, iters: int, seed: int, sample: int | None = None):
    """Plain Lloyd k-means on CPU (FP64) -> assignment of every row.

    Only an input helper for small test workloads: the IVF partition is an
    input of the method (Section 4.1 uses KMeans without fixing it), so the
    oracle and the GPU path both receive the same assignment.
    """
    g = rng(seed)
    Xs = X if sample is None or sample >= len(X) else X[g.choice(len(X), size=sample, replace=False)]
    C = Xs[g.choice(len(Xs), size=nlist, replace=False)].astype(np.float64)
    Xs64 = Xs.astype(np.float64)
    for _ in range(iters):
        d2 = (Xs64 ** 2).sum(1)[:, None] - 2 * Xs64 @ C.T + (C ** 2).sum(1)[None, :]
        a = d2.argmin(1)
        for j in range(nlist):
            m = a == j
            if m.any():
                C[j] = Xs64[m].mean(0)
    X64 = X.astype(np.float64)
    out = np.empty(len(X), dtype=np.int32)
    for s0 in range(0, len(X), 1 << 14):
        blk = X64[s0:s0 + (1 << 14)]
        d2 = (blk ** 2).sum(1)[:, None] - 2 * blk @ C.T + (C ** 2).sum(1)[None, :]
        out[s0:s0 + len(blk)] = d2.argmin(1)
    return out


def kmeans_assign_torch(X, nlist: int, iters: int, seed: int, sample: int | None = None, device=None,
                        chunk: int = 32768):
    """Lloyd k-means with plain torch ops (runs on ``device``, GPU if given),
    returning the cluster of every row (int32 numpy).  An input generator for
    the IVF partition at million scale, where the numpy version is too slow;
    it is not part of the method and not part of the library under test."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    g = rng(seed)
    n = len(X)
    idx = np.sort(g.choice(n, size=sample, replace=False)) if sample and sample < n else np.arange(n)
    Xs = torch.from_numpy(np.ascontiguousarray(X[idx])).to(dev)
    C = Xs[torch.from_numpy(g.choice(len(idx), size=nlist, replace=False)).to(dev)].clone()
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False

    def assign(rows):
        out = torch.empty(len(rows), dtype=torch.int64, device=dev)
        cn = (C * C).sum(1)
        for s0 in range(0, len(rows), chunk):
            b = rows[s0:s0 + chunk]
            d = cn[None, :] - 2.0 * (b @ C.T)
            out[s0:s0 + len(b)] = d.argmin(1)
        return out

    try:
        for _ in range(iters):
            a = assign(Xs)
            sums = torch.zeros_like(C).index_add_(0, a, Xs)
            cnt = torch.bincount(a, minlength=nlist).to(C.dtype)
            nz = cnt > 0
            C[nz] = sums[nz] / cnt[nz, None]
        out = np.empty(n, dtype=np.int32)
        for s0 in range(0, n, 1 << 18):
            blk = torch.from_numpy(np.ascontiguousarray(X[s0:s0 + (1 << 18)])).to(dev)
            out[s0:s0 + len(blk)] = assign(blk).cpu().numpy()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


# The five workloads (sizes, bit widths and query mixes).  Names describe the
# workload; ``role`` says what each is used for.
WORKLOADS = {
    "bruteforce_n10k_d128_b4": dict(
        n=10_000, d=128, n_comp=16, scale="unit", nq=100, B=4, nlist=1,
        k=10, rerank_k=100, data_seed=0, query_seed=1, p_seed=7),
    "ivf_n1m_d960_nlist4096": dict(
        n=1_000_000, d=960, n_comp=256, scale="aniso", nq=10_000, B=5, Bs=(3, 5, 7),
        nlist=4096, nprobes=(16, 32, 64, 128, 256), k=10, data_seed=0, query_seed=1,
        p_seed=7, kmeans_iters=10, kmeans_sample=262_144),
    "embed_n2m_d1536_b7": dict(
        n=2_000_000, d=1536, n_comp=512, scale="unit", normalize=True, nq=10_000, B=7,
        nlist=4096, nprobe=64, k=10, data_seed=0, query_seed=1, p_seed=7),
    "zipf_n5m_d768_nlist8192": dict(
        n=5_000_000, d=768, n_comp=8192, scale="unit", zipf_s=1.1, nq=16_384, B=5,
        nlist=8192, nprobe_lo=8, nprobe_hi=256, ks=(10, 100), data_seed=0,
        query_seed=1, p_seed=7, nprobe_seed=3),
    "backward_n1m_d1024_b4": dict(
        n=1_000_000, d=1024, n_comp=256, scale="aniso", nq=4096, B=4, nlist=4096,
        nprobe=64, k=100, data_seed=0, query_seed=1, p_seed=7, grad_seed=2),
}
