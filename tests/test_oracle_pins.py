"""Pins the CPU oracle for windowed aggregation to things other than itself.

* hand-worked micro-streams (tests/golden/window_semantics.json);
* brute force: every (window, key) recomputed from the full event log with numpy;
* closed forms / invariants: sum of counts = K * surviving events (every
  surviving event lies in exactly size/slide windows), per-key totals equal
  numpy.bincount, a tumbling window over the whole stream equals a plain
  group-by (numpy.bincount / minimum.at / maximum.at);
* batching invariance for in-order streams.
Semantics follow the event-time window definition written at the top of
oracle/window_agg_oracle.cpp (the paper, Table I/III, names tumbling and
sliding windows with SUM/AVG group-bys but leaves their semantics to Spark).
"""
import json
import os

import numpy as np
import pytest

from oracle import window_agg as wa
from paper_2111_04289_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "window_semantics.json")
COLS = {"ts": wa.COL_TS, "key": wa.COL_KEY, "value": wa.COL_VALUE, "type": wa.COL_TYPE}
OPS = {"none": wa.OP_NONE, "eq": wa.OP_EQ, "ne": wa.OP_NE, "lt": wa.OP_LT,
       "le": wa.OP_LE, "gt": wa.OP_GT, "ge": wa.OP_GE}


def _rows_as_tuples(rows, is_float):
    out = []
    for r in rows:
        if is_float:
            out.append((int(r["window_start"]), int(r["window_end"]), int(r["key"]),
                        int(r["count"]), float(r["sum_f"]), float(r["min_f"]),
                        float(r["max_f"]), float(r["avg"])))
        else:
            out.append((int(r["window_start"]), int(r["window_end"]), int(r["key"]),
                        int(r["count"]), int(r["sum_i"]), int(r["min_i"]),
                        int(r["max_i"]), float(r["avg"])))
    return out


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_micro_streams(case):
    is_float = case["value_type"] == "float32"
    o = wa.WindowAggOracle(is_float, case["lateness"])
    q = case["query"]
    fc, fo, fv = COLS[q["filter_col"]], OPS[q["filter_op"]], q["filter"]
    qid = o.add_query(fc, fo, int(fv) if not isinstance(fv, float) else 0,
                      float(fv), q["size"], q["slide"])
    for push in case["pushes"]:
        rows = push["rows"]
        ts = np.array([r[0] for r in rows], dtype=np.int64)
        key = np.array([r[1] for r in rows], dtype=np.uint32)
        val = np.array([r[2] for r in rows], dtype=np.float32 if is_float else np.int32)
        typ = np.array([r[3] for r in rows], dtype=np.uint8)
        o.push(ts, key, val, typ, eos=push["eos"])
        got = o.take_rows(qid)
        exp = push["expect"]
        assert len(got) == len(exp), (case["name"], got, exp)
        for g, e in zip(_rows_as_tuples(got, is_float), exp):
            assert g[:4] == tuple(e[:4])
            if is_float:
                assert g[4] == e[4] and g[7] == e[7]
                # min/max compared bitwise so that -0.0 and +0.0 differ
                assert np.float32(g[5]).tobytes() == np.float32(e[5]).tobytes()
                assert np.float32(g[6]).tobytes() == np.float32(e[6]).tobytes()
            else:
                assert g[4:7] == tuple(e[4:7]) and g[7] == e[7]
        assert o.late_rows(qid) == push["late"]


# --------------------------------------------------------------------------- #
# brute force
# --------------------------------------------------------------------------- #

def _filter_mask(b: synth.Batch, col, op, fi, ff, is_float):
    if op == wa.OP_NONE:
        return np.ones(len(b), dtype=bool)
    if col == wa.COL_TS:
        x, c = b.ts.astype(np.int64), fi
    elif col == wa.COL_KEY:
        x, c = b.key.astype(np.int64), fi
    elif col == wa.COL_TYPE:
        x, c = b.type.astype(np.int64), fi
    else:
        x, c = (b.value.astype(np.float64), ff) if is_float else (b.value.astype(np.int64), fi)
    return {wa.OP_EQ: x == c, wa.OP_NE: x != c, wa.OP_LT: x < c, wa.OP_LE: x <= c,
            wa.OP_GT: x > c, wa.OP_GE: x >= c}[op]


def brute_force(b: synth.Batch, size, slide, mask, is_float):
    """All (window, key) aggregates from the complete event log (no state)."""
    ts, key, val = b.ts[mask], b.key[mask], b.value[mask]
    if ts.size == 0:
        return []
    lo = (int(ts.min()) // slide - size // slide) * slide
    hi = int(ts.max())
    rows = []
    for s in range(lo, hi + 1, slide):
        sel = (ts >= s) & (ts < s + size)
        if not sel.any():
            continue
        k, v = key[sel], val[sel]
        for kk in np.unique(k):
            vv = v[k == kk]
            if is_float:
                ssum = float(np.sum(vv.astype(np.float64)))
                rows.append((s, s + size, int(kk), int(vv.size), ssum, float(vv.min()),
                             float(vv.max()), ssum / vv.size))
            else:
                ssum = int(np.sum(vv.astype(np.int64)))
                rows.append((s, s + size, int(kk), int(vv.size), ssum, int(vv.min()),
                             int(vv.max()), ssum / vv.size))
    return rows


def _run_oracle(batches, size, slide, col, op, fi, ff, is_float, lateness=0):
    o = wa.WindowAggOracle(is_float, lateness)
    qid = o.add_query(col, op, fi, ff, size, slide)
    out = []
    for i, b in enumerate(batches):
        o.push(b.ts, b.key, b.value, b.type, eos=(i == len(batches) - 1))
        out.extend(_rows_as_tuples(o.take_rows(qid), is_float))
    return out, o.late_rows(qid)


def _concat(batches):
    return synth.Batch(
        np.concatenate([b.ts for b in batches]), np.concatenate([b.key for b in batches]),
        np.concatenate([b.value for b in batches]),
        None if batches[0].type is None else np.concatenate([b.type for b in batches]),
    )


def _compare(got, exp, is_float):
    assert len(got) == len(exp)
    for g, e in zip(got, exp):
        assert g[:4] == e[:4]
        if is_float:
            assert g[4] == pytest.approx(e[4], rel=1e-12, abs=0)
            assert g[5:7] == e[5:7]
            assert g[7] == pytest.approx(e[7], rel=1e-12, abs=0)
        else:
            assert g[4:8] == e[4:8]


@pytest.mark.parametrize("size,slide", [(10_000, 10_000), (60_000, 5_000), (3_000, 1_000), (7, 7)])
def test_brute_force_int_stream(size, slide):
    s = synth.TinyIntStream(seed=11, card=37)
    batches = [s.next_batch(n) for n in (700, 1, 0, 1300, 333)]
    got, late = _run_oracle(batches, size, slide, wa.COL_TYPE, wa.OP_EQ, 0, 0.0, False)
    allb = _concat(batches)
    mask = _filter_mask(allb, wa.COL_TYPE, wa.OP_EQ, 0, 0.0, False)
    _compare(got, brute_force(allb, size, slide, mask, False), False)
    assert late == 0


@pytest.mark.parametrize("size,slide", [(60_000, 5_000), (1_000, 1_000)])
def test_brute_force_float_stream(size, slide):
    s = synth.LargeFloatStream(seed=12, card=500, s=1.1)
    batches = [s.next_batch(n) for n in (900, 1100, 17)]
    got, late = _run_oracle(batches, size, slide, wa.COL_VALUE, wa.OP_GT, 0, 0.5, True)
    allb = _concat(batches)
    mask = _filter_mask(allb, wa.COL_VALUE, wa.OP_GT, 0, 0.5, True)
    _compare(got, brute_force(allb, size, slide, mask, True), True)
    assert late == 0


def test_brute_force_jittered_stream_with_allowance():
    """Out-of-order by <= 5 ms with 5 ms allowed lateness: nothing is late."""
    rng = np.random.default_rng(13)
    s = synth.TinyIntStream(seed=13, card=50)
    batches = []
    for n in (500, 800, 600):
        b = s.next_batch(n)
        b.ts = synth.jitter_ts(rng, b.ts, 5)
        batches.append(b)
    got, late = _run_oracle(batches, 2_000, 500, wa.COL_TS, wa.OP_NONE, 0, 0.0, False,
                            lateness=5)
    allb = _concat(batches)
    mask = np.ones(len(allb), dtype=bool)
    assert late == 0
    _compare(got, brute_force(allb, 2_000, 500, mask, False), False)


# --------------------------------------------------------------------------- #
# invariants and library special cases
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("size,slide", [(60_000, 5_000), (30_000, 1_000), (10_000, 10_000)])
def test_each_event_lands_in_size_over_slide_windows(size, slide):
    s = synth.TinyIntStream(seed=21, card=1024)
    batches = [s.next_batch(4096) for _ in range(3)]
    got, _ = _run_oracle(batches, size, slide, wa.COL_TYPE, wa.OP_EQ, 0, 0.0, False)
    allb = _concat(batches)
    mask = allb.type == 0
    K = size // slide
    counts = np.array([g[3] for g in got], dtype=np.int64)
    sums = np.array([g[4] for g in got], dtype=np.int64)
    assert counts.sum() == K * int(mask.sum())
    assert sums.sum() == K * int(allb.value[mask].astype(np.int64).sum())
    # per key: sum over windows of count = K * bincount
    keys = np.array([g[2] for g in got], dtype=np.int64)
    per_key = np.bincount(keys, weights=counts, minlength=1024)
    np.testing.assert_array_equal(per_key, K * np.bincount(allb.key[mask], minlength=1024))


def test_single_window_is_plain_group_by():
    s = synth.LargeFloatStream(seed=22, card=300, s=1.1)
    batches = [s.next_batch(1500), s.next_batch(1500)]
    span = int(batches[-1].ts[-1]) + 1  # all ts in [0, span)
    got, _ = _run_oracle(batches, span, span, wa.COL_TS, wa.OP_NONE, 0, 0.0, True)
    allb = _concat(batches)
    assert all(g[0] == 0 for g in got)
    k = allb.key.astype(np.int64)
    cnt = np.bincount(k, minlength=300)
    ssum = np.bincount(k, weights=allb.value.astype(np.float64), minlength=300)
    mn = np.full(300, np.inf, dtype=np.float32)
    mx = np.full(300, -np.inf, dtype=np.float32)
    np.minimum.at(mn, k, allb.value)
    np.maximum.at(mx, k, allb.value)
    present = np.nonzero(cnt)[0]
    assert [g[2] for g in got] == list(present)
    for g in got:
        kk = g[2]
        assert g[3] == cnt[kk]
        assert g[4] == pytest.approx(ssum[kk], rel=1e-12)
        assert g[5] == mn[kk] and g[6] == mx[kk]


@pytest.mark.parametrize("cuts", [[4000], [1000, 3000], [1, 2, 3997], [2000, 0, 2000]])
def test_batching_invariance(cuts):
    s = synth.TinyIntStream(seed=23, card=64)
    full = s.next_batch(4000)
    ref, _ = _run_oracle([full, full.slice(0, 0)], 20_000, 2_000, wa.COL_TS, wa.OP_NONE,
                         0, 0.0, False)
    pieces, a = [], 0
    for c in cuts:
        pieces.append(full.slice(a, a + c))
        a += c
    pieces.append(full.slice(a, 4000))
    got, _ = _run_oracle(pieces, 20_000, 2_000, wa.COL_TS, wa.OP_NONE, 0, 0.0, False)
    assert got == ref


def test_emission_respects_watermark():
    """After each batch every emitted window has end <= wm, every open one end > wm."""
    s = synth.TinyIntStream(seed=24, card=16)
    o = wa.WindowAggOracle(False, 0)
    qid = o.add_query(wa.COL_TS, wa.OP_NONE, 0, 0.0, 3_000, 1_000)
    wm = None
    last_start = None
    for _ in range(6):
        b = s.next_batch(900)
        o.push(b.ts, b.key, b.value, b.type)
        wm = int(b.ts.max()) if wm is None else max(wm, int(b.ts.max()))
        rows = o.take_rows(qid)
        assert np.all(rows["window_end"] <= wm)
        starts = rows["window_start"]
        if rows.size:
            assert np.all(np.diff(starts) >= 0)
            if last_start is not None:
                assert starts[0] > last_start
            last_start = int(starts[-1])
    # what is still open ends after the watermark: emitted at end of stream
    o.push(np.zeros(0, np.int64), np.zeros(0, np.uint32), np.zeros(0, np.int32), None, eos=True)
    rows = o.take_rows(qid)
    assert np.all(rows["window_end"] > wm)


# --------------------------------------------------------------------------- #
# post-aggregation: GROUP BY packed key fields, HAVING, ORDER BY (Table III)
# --------------------------------------------------------------------------- #

def _brute_groups(ts, key, val, size, slide, mask):
    """{(window start, key & mask): (count, sum, min, max)} from the events."""
    K = size // slide
    out = {}
    for t, k, v in zip(ts.tolist(), (key & np.uint32(mask)).tolist(), val.tolist()):
        w0 = t // slide
        for j in range(K):
            g = ((w0 - j) * slide, k)
            c, s, mn, mx = out.get(g, (0, 0, None, None))
            out[g] = (c + 1, s + v, v if mn is None else min(mn, v), v if mx is None else max(mx, v))
    return out


def _three_field_stream(seed, n=3000):
    """Key = highway (4 bits) | direction (1 bit) << 4 | segment (7 bits) << 5,
    int speeds 0..120 (the LR2S query's shape)."""
    rng = np.random.default_rng(seed)
    hw, dr, sg = rng.integers(0, 3, n), rng.integers(0, 2, n), rng.integers(0, 20, n)
    key = (hw | (dr << 4) | (sg << 5)).astype(np.uint32)
    ts = np.sort(rng.integers(0, 9000, n)).astype(np.int64)
    val = rng.integers(0, 121, n).astype(np.int32)
    return ts, key, val


@pytest.mark.parametrize("mask", [0xFFFFFFFF, 0b11111, 0b111111100000, 0b1111])
def test_group_by_key_fields_equals_brute_force(mask):
    ts, key, val = _three_field_stream(5)
    o = wa.WindowAggOracle(False, 0)
    q = o.add_query(size_ms=3000, slide_ms=1000)
    o.set_post(q, group_mask=mask)
    o.push(ts, key, val, None, eos=True)
    rows = o.take_rows(q)
    exp = _brute_groups(ts, key, val, 3000, 1000, mask)
    assert len(rows) == len(exp)
    assert all(int(r["key"]) & ~mask & 0xFFFFFFFF == 0 for r in rows)
    for r in rows:
        c, s, mn, mx = exp[(int(r["window_start"]), int(r["key"]))]
        assert (int(r["count"]), int(r["sum_i"]), int(r["min_i"]), int(r["max_i"])) == (c, s, mn, mx)


@pytest.mark.parametrize("having", [("avg", wa.OP_LT, 40.0), ("count", wa.OP_GE, 30),
                                    ("max", wa.OP_EQ, 120), ("sum", wa.OP_NE, 0)])
def test_having_keeps_the_rows_whose_aggregate_passes(having):
    """LR2S: ... GROUPBY (highway, direction, segment) HAVING avgSpeed < 40."""
    ts, key, val = _three_field_stream(6)
    o = wa.WindowAggOracle(False, 0)
    q = o.add_query(size_ms=3000, slide_ms=1000)
    o.set_post(q, group_mask=0b111111111111, having=having)
    o.push(ts, key, val, None, eos=True)
    rows = o.take_rows(q)
    agg, op, c = having
    pick = {"count": 0, "sum": 1, "min": 2, "max": 3}
    test = {wa.OP_LT: np.less, wa.OP_GE: np.greater_equal, wa.OP_EQ: np.equal,
            wa.OP_NE: np.not_equal}[op]
    exp = sorted(g for g, a in _brute_groups(ts, key, val, 3000, 1000, 0xFFF).items()
                 if test(a[1] / a[0] if agg == "avg" else a[pick[agg]], c))
    assert [(int(r["window_start"]), int(r["key"])) for r in rows] == exp


@pytest.mark.parametrize("agg,desc", [("sum", False), ("sum", True), ("count", True),
                                      ("min", False)])
def test_order_by_sorts_each_window_by_the_aggregate(agg, desc):
    """CM1: ... GROUPBY category ORDERBY SUM(cpu): per window, rows sorted by
    the aggregate, equal values in key order (numpy.lexsort on (key, value))."""
    rng = np.random.default_rng(7)
    n = 4000
    ts = np.sort(rng.integers(0, 20_000, n)).astype(np.int64)
    key = rng.integers(0, 30, n).astype(np.uint32)
    val = rng.integers(0, 5, n).astype(np.int32)  # many equal aggregates
    o = wa.WindowAggOracle(False, 0)
    q = o.add_query(size_ms=6000, slide_ms=2000)
    o.set_post(q, order_by=(agg, desc))
    o.push(ts[: n // 2], key[: n // 2], val[: n // 2], None)
    o.push(ts[n // 2:], key[n // 2:], val[n // 2:], None, eos=True)
    rows = o.take_rows(q)
    exp = _brute_groups(ts, key, val, 6000, 2000, 0xFFFFFFFF)
    pick = {"count": 0, "sum": 1, "min": 2, "max": 3}[agg]
    starts = sorted({g[0] for g in exp})
    expected = []
    for w in starts:
        ks = np.array(sorted(k for (s, k) in exp if s == w), dtype=np.int64)
        vs = np.array([exp[(w, int(k))][pick] for k in ks], dtype=np.int64)
        order = np.lexsort((ks, -vs if desc else vs))
        expected += [(w, int(k)) for k in ks[order]]
    assert [(int(r["window_start"]), int(r["key"])) for r in rows] == expected


# --------------------------------------------------------------------------- #
# windowed equi-join (LR1S / LR1T of Table III): explicit pair enumeration
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("size,slide", [(100, 100), (90, 30)])
def test_window_join_equals_enumerated_pairs(size, slide):
    from oracle import join as oj
    rng = np.random.default_rng(11)
    n = 300
    ts = np.sort(rng.integers(0, 400, n)).astype(np.int64)
    key = rng.integers(0, 12, n).astype(np.uint32)
    val = rng.integers(-5, 50, n).astype(np.int32)
    typ = rng.integers(0, 2, n).astype(np.uint8)
    left = (wa.COL_TYPE, wa.OP_EQ, 0, 0.0)
    right = (wa.COL_TYPE, wa.OP_EQ, 1, 0.0)
    o = oj.WindowJoinOracle(False, size, slide, left, right)
    rows = np.concatenate([o.push(ts[:150], key[:150], val[:150], typ[:150]),
                           o.push(ts[150:], key[150:], val[150:], typ[150:], eos=True)])
    o.close()
    # every window any event lies in; every (left, right) event pair with equal keys
    K = size // slide
    exp = {}
    for a in range(n):
        if typ[a] != 0:
            continue
        for b in range(n):
            if typ[b] != 1 or key[a] != key[b]:
                continue
            wa_ = {(ts[a] // slide - j) * slide for j in range(K)}
            wb_ = {(ts[b] // slide - j) * slide for j in range(K)}
            for w in wa_ & wb_:  # both events in window w
                p, sl, sr = exp.get((w, int(key[a])), (0, 0, 0))
                exp[(w, int(key[a]))] = (p + 1, sl + int(val[a]), sr + int(val[b]))
    assert len(rows) == len(exp) > 0
    for r in rows:
        p, sl, sr = exp[(int(r["window_start"]), int(r["key"]))]
        assert int(r["pairs"]) == p
        # per-pair sums: sum of l.value over pairs = left_sum * right_count
        assert r["left_sum"] * r["right_count"] == sl and r["right_sum"] * r["left_count"] == sr
    keys = [(int(r["window_start"]), int(r["key"])) for r in rows]
    assert keys == sorted(keys)


def test_self_join_pairs_are_squared_counts():
    """LR1: a stream joined with itself on vehicle: pairs = count^2 per window."""
    from oracle import join as oj
    b = synth.TinyIntStream(seed=12, card=15).next_batch(2000)
    allrows = (wa.COL_TS, wa.OP_NONE, 0, 0.0)
    o = oj.WindowJoinOracle(False, 3000, 1000, allrows, allrows)
    rows = o.push(b.ts, b.key, b.value, b.type, eos=True)
    o.close()
    assert len(rows) > 0
    assert np.array_equal(rows["pairs"], rows["left_count"] ** 2)
    assert np.array_equal(rows["left_count"], rows["right_count"])
