"""Host checks of the tensor-core scan's admission bound (no GPU).

The scan's filter warps first vote on a relaxed threshold on the raw tile
value v = g + (f_res/2) acc, thr = (tf - dq) + (2^-20 (|tf| + |dq|) + 2^-120)
(`relaxed_threshold` in k_scan_tc.cu), and only then apply the float test
fl(dq + v) <= tf and the exact key test.  A candidate is lost if the relaxed
test ever rejects a value the float test admits, so the relaxed test must be
a superset of the float test for every FP32 input: checked here in IEEE
single precision (numpy float32, round to nearest) on values at and around
the boundary, across magnitudes, signs, zeros, subnormals and +inf."""
import numpy as np

F = np.float32


def _relaxed(tf, dq):
    with np.errstate(over="ignore", invalid="ignore"):
        return (tf - dq) + (F(2.0 ** -20) * (np.abs(tf) + np.abs(dq)) + F(2.0 ** -120))


def _admitted_by_float_test(v, dq, tf):
    with np.errstate(over="ignore", invalid="ignore"):
        return (dq + v) <= tf


def _boundary_values(tf, dq, steps=48):
    """v around fl(tf - dq), walked ulp by ulp in both directions."""
    with np.errstate(over="ignore", invalid="ignore"):
        v0 = (tf - dq).astype(F)
    out = [v0]
    up = v0.copy()
    dn = v0.copy()
    for _ in range(steps):
        up = np.nextafter(up, F(np.inf))
        dn = np.nextafter(dn, F(-np.inf))
        out += [up, dn]
    return np.stack(out, 1)


def _check(tf, dq):
    tf = np.asarray(tf, F)
    dq = np.asarray(dq, F)
    thr = _relaxed(tf, dq)[:, None]
    v = _boundary_values(tf, dq)
    ok = np.isfinite(v)
    adm = _admitted_by_float_test(v, dq[:, None], tf[:, None]) & ok
    bad = adm & ~(v <= thr)
    assert not bad.any(), (tf[bad.any(1)][:5], dq[bad.any(1)][:5])
    return int(adm.sum())


def test_relaxed_threshold_admits_every_float_admission_random_magnitudes():
    g = np.random.default_rng(91)
    n = 20000
    total = 0
    for lo, hi in ((-3, 3), (-20, 20), (-38, 38)):
        mag_t = 10.0 ** g.uniform(lo, hi, n)
        mag_d = 10.0 ** g.uniform(lo, hi, n)
        tf = (mag_t * g.choice([-1.0, 1.0], n)).astype(F)
        dq = (mag_d * g.choice([-1.0, 1.0], n)).astype(F)
        total += _check(tf, dq)
    assert total > 100000          # the boundary walk admits about half of its values


def test_relaxed_threshold_distance_like_values():
    """Squared distances and their parts as the search forms them: dq =
    ||q_r - c||^2 >= 0, tf a k'-th estimate of similar size."""
    g = np.random.default_rng(92)
    n = 50000
    dq = (g.gamma(4.0, 50.0, n)).astype(F)
    tf = (dq * g.uniform(0.5, 2.0, n) + g.normal(0, 5, n)).astype(F)
    assert _check(tf, dq) > 100000


def test_relaxed_threshold_special_values():
    tiny = np.float32(1e-45)                     # smallest subnormal
    sub = np.float32(3e-39)
    big = np.float32(3e38)
    cases = [(0.0, 0.0), (tiny, 0.0), (0.0, tiny), (-tiny, tiny), (sub, -sub), (sub, sub),
             (big, -big / 4), (-big, big / 4), (1.0, 1.0), (1.0, -1.0), (-1.0, 1.0), (1e-30, 1e30),
             (1e30, 1e-30), (np.float32(2.0 ** -126), np.float32(2.0 ** -127))]
    tf = np.array([c[0] for c in cases], F)
    dq = np.array([c[1] for c in cases], F)
    _check(tf, dq)
    # an empty list's threshold (+inf) admits every finite value
    thr = _relaxed(np.array([np.inf], F), np.array([123.0], F))
    assert np.isinf(thr[0]) and thr[0] > 0
    # a NaN tile value (rows past a block's end) is admitted by neither test
    nan = np.float32(np.nan)
    assert not (nan <= _relaxed(np.array([5.0], F), np.array([1.0], F))[0])
    assert not _admitted_by_float_test(nan, F(1.0), F(np.inf))
