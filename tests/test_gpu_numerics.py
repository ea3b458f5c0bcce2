"""GPU numerics of float sums whose values do not share a sign, and of
averages of groups that hold an infinity among more than 2^24 events.

Validity criterion for a float sum (also stated in the design doc): with n the
row's count, M = max |v| (from the oracle's min and max) and S1 = sum |v|
(the oracle run on |v|),

    |engine - oracle| <= 1e-9 |oracle| + 4 (n + 1) 2^-53 S1 + n 2^-52 M.

The last term bounds the fused pass's fixed-point rounding (every value is
rounded to a unit of at most 2^-52 of the largest |value| of its group in
its tile); the middle one bounds, to first order, the reassociation error of
both FP64 summations (the oracle's sequential one and the engine's tree of
partial sums, each of depth <= n + 1, each addition off by at most 2^-53 of a
partial sum bounded by S1).  For values of one sign S1 = |sum| and the
criterion is the 1e-9 relative tolerance of the other tests.
"""
import numpy as np
import pytest

from paper_2111_04289_b300 import synth
from tests.engine_helpers import run_engine, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mixed_sign_batches(seed):
    rng = np.random.default_rng(seed)
    n = 200_000
    key = rng.integers(0, 64, n).astype(np.uint32)
    mag = rng.lognormal(0.0, 2.0, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    val = (mag * sign).astype(np.float32)
    # keys 0..7: every value followed by its negation somewhere in the same
    # window, so the exact sum is 0
    for k in range(8):
        idx = np.flatnonzero(key == k)
        half = len(idx) // 2
        val[idx[half:2 * half]] = -val[idx[:half]]
        if len(idx) % 2:
            val[idx[-1]] = 0.0
    ts = np.sort(rng.integers(0, 40_000, n)).astype(np.int64)
    b = synth.Batch(ts, key, val)
    return [b.slice(0, n // 3), b.slice(n // 3, n)]


@pytest.mark.parametrize("window", [dict(size=40_000), dict(size=8_000, slide=2_000)])
def test_mixed_sign_sums_within_the_stated_bound(window):
    batches = _mixed_sign_batches(81)
    q = [window]
    eng, _ = run_engine(batches, q, True, torch=torch)
    orc, _ = run_oracle(batches, q, True)
    absb = [synth.Batch(b.ts, b.key, np.abs(b.value)) for b in batches]
    s1, _ = run_oracle(absb, q, True)
    e, o, a = eng[0], orc[0], s1[0]
    assert len(e) == len(o) == len(a) > 0
    for f in ("window_start", "key", "count"):
        np.testing.assert_array_equal(e[f], o[f])
    np.testing.assert_array_equal(e["min"].view(np.uint32), o["min_f"].view(np.uint32))
    np.testing.assert_array_equal(e["max"].view(np.uint32), o["max_f"].view(np.uint32))
    n = o["count"].astype(np.float64)
    m = np.maximum(np.abs(o["min_f"].astype(np.float64)), np.abs(o["max_f"].astype(np.float64)))
    tol = 1e-9 * np.abs(o["sum_f"]) + 4 * (n + 1) * 2.0**-53 * a["sum_f"] + n * 2.0**-52 * m
    err = np.abs(e["sum"] - o["sum_f"])
    assert np.all(err <= tol), float(np.max(err / tol))
    # cancelling keys really cancel far below their magnitude
    cancel = e["key"] < 8
    if window.get("slide") is None:
        assert np.all(np.abs(e["sum"][cancel]) <= tol[cancel])
    avg_tol = tol / n
    assert np.all(np.abs(e["avg"] - o["avg"]) <= avg_tol * (1 + 1e-12) + 1e-300)


@pytest.mark.parametrize("inf", [np.inf, -np.inf])
def test_infinite_value_among_more_than_2p24_events(inf):
    """A key holding one infinity among 2^24 + 1 events (counts from 2^24 on
    divide by a refined float32 reciprocal): its sum and average are that
    infinity (the definition: Inf / n), min or max is it too; a second key
    with 2^24 + 3 finite events stays finite."""
    rng = np.random.default_rng(83)
    n1, n2 = (1 << 24) + 1, (1 << 24) + 3
    key = np.concatenate([np.full(n1, 3, np.uint32), np.full(n2, 4, np.uint32)])
    val = rng.lognormal(0.0, 1.0, n1 + n2).astype(np.float32)
    val[12345] = np.float32(inf)
    perm = rng.permutation(n1 + n2)
    key, val = key[perm], val[perm]
    ts = np.sort(rng.integers(0, 1000, n1 + n2)).astype(np.int64)
    eng, _ = run_engine([synth.Batch(ts, key, val)], [dict(size=1000)], True, device_input=True,
                        torch=torch)
    e = eng[0]
    assert e["key"].tolist() == [3, 4]
    assert e["count"].tolist() == [n1, n2]
    assert e["sum"][0] == inf and e["avg"][0] == inf
    assert (e["max"][0] == inf) if inf > 0 else (e["min"][0] == inf)
    v4 = val[key == 4].astype(np.float64)
    import math
    exact = math.fsum(v4)
    assert abs(e["sum"][1] - exact) <= 1e-9 * exact
    assert abs(e["avg"][1] - exact / n2) <= 1e-9 * exact / n2
