"""Key-sharded streams and snapshot / resume on the GPU, against one unsharded
oracle stream.

* ShardedStream over 1-4 engine streams (all on cuda:0 here: independent
  streams, no kernel waits on another) gives, merged, the oracle's rows of a
  single stream: same windows, keys, counts, min / max, int sums exactly,
  float sums within the engine's float tolerance.
* The watermark hint: an empty push with lms_stream_set_batch_max_ts closes
  what an oracle push with that max event time closes.
* lms_stream_snapshot / lms_stream_restore: a stream snapshotted between
  batches (rows still unpolled, windows still open, a join registered),
  closed, and restored continues exactly as the oracle's uninterrupted run.
"""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import sharded
from tests.shard_helpers import OracleShard
from tests.test_sharded_cpu import QUERIES, _batches, _run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLOAT_REL_TOL = 1e-9


def _same(a, e, is_float, ctx):
    assert len(a) == len(e), ctx
    for f in ("window_start", "key", "count"):
        np.testing.assert_array_equal(a[f], e[f], err_msg=ctx)
    if is_float:
        np.testing.assert_array_equal(a["min"].view(np.uint32), e["min"].view(np.uint32))
        np.testing.assert_array_equal(a["max"].view(np.uint32), e["max"].view(np.uint32))
        for f in ("sum", "avg"):
            assert np.all(np.abs(a[f] - e[f]) <= FLOAT_REL_TOL * np.abs(e[f]) + 1e-300), ctx
    else:
        for f in ("sum", "min", "max"):
            np.testing.assert_array_equal(a[f], e[f], err_msg=ctx)
        np.testing.assert_array_equal(a["avg"].view(np.uint64), e["avg"].view(np.uint64))


def _same_join(a, e, is_float, ctx):
    assert len(a) == len(e), ctx
    for f in ("window_start", "key", "pairs", "left_count", "right_count"):
        np.testing.assert_array_equal(a[f], e[f], err_msg=ctx)
    for f in ("left_sum", "right_sum"):
        x, y = a[f].astype(np.float64), e[f].astype(np.float64)
        assert np.all(np.abs(x - y) <= FLOAT_REL_TOL * np.abs(y) + 1e-300), ctx


def _queries_for(is_float):
    # an ORDER BY on a float sum could flip the order of two nearly equal sums
    # within tolerance; the value-ordered queries run on int streams
    return QUERIES if not is_float else [q for q in QUERIES if "order_by" not in q]


@pytest.mark.parametrize("g", [1, 2, 4])
@pytest.mark.parametrize("float_values", [False, True])
def test_sharded_engine_streams_equal_one_oracle_stream(g, float_values):
    vt = "float32" if float_values else "int32"
    queries = _queries_for(float_values)
    batches = _batches(41 + g, n=20000, card=3000, float_values=float_values, lateness_jitter=40)
    kw = dict(value_type=vt, has_type=True, allowed_lateness_ms=25, key_fields=(8, 8))
    ref_rows, ref_join = _run(OracleShard(**kw), batches, queries)
    sh = sharded.ShardedStream.open(g, devices=[0] * g, key_mask=0xFF, **kw)
    try:
        got_rows, got_join = _run(sh, batches, queries)
    finally:
        sh.close()
    for q in range(len(queries)):
        for b in range(len(batches)):
            _same(got_rows[q][b], ref_rows[q][b], float_values, f"q{q} b{b}")
    for b in range(len(batches)):
        _same_join(got_join[b], ref_join[b], float_values, f"join b{b}")
    assert sum(len(r) for r in ref_rows[0]) > 1000


def test_watermark_hint_closes_windows_of_an_empty_push():
    rng = np.random.default_rng(7)
    n = 5000
    ts = np.sort(rng.integers(0, 3000, n)).astype(np.int64)
    key = rng.integers(0, 50, n).astype(np.uint32)
    val = rng.integers(-100, 100, n).astype(np.int32)
    s = lm.Stream("int32")
    o = OracleShard("int32")
    for x in (s, o):
        x.register_query(1000)
        x.register_query(1000, 250)
    s.push(ts, key, val)
    o.push(ts, key, val)
    e0 = [s.poll(0), s.poll(1)]
    r0 = [o.poll(0), o.poll(1)]
    for x in (s, o):
        x.set_batch_max_ts(5200)
        x.push(ts[:0], key[:0], val[:0])
    e1 = [s.poll(0), s.poll(1)]
    r1 = [o.poll(0), o.poll(1)]
    assert s.stats()["watermark"] == 5200
    with pytest.raises(lm.LmsError):
        s.set_origin(0)  # the origin is fixed by the first push
    s.close()
    for a, e in zip(e0 + e1, r0 + r1):
        _same(a, e, False, "hint")
    # the first push closed the tumbling windows before 2000; the hint closes [2000, 3000)
    assert len(e1[0]) > 0 and set(e1[0]["window_start"].tolist()) == {2000}


@pytest.mark.parametrize("float_values", [False, True])
def test_snapshot_restore_continues_like_an_uninterrupted_stream(float_values):
    vt = "float32" if float_values else "int32"
    queries = _queries_for(float_values)
    batches = _batches(53, n=30000, card=5000, float_values=float_values, lateness_jitter=40)
    kw = dict(value_type=vt, has_type=True, allowed_lateness_ms=25, key_fields=(8, 8))
    ref_rows, ref_join = _run(OracleShard(**kw), batches, queries)
    s = lm.Stream(vt, has_type=True, allowed_lateness_ms=25, key_fields=(8, 8))
    qids = [s.register_query(**q) for q in queries]
    jid = s.register_join(400, 200, ("type", "eq", 0), ("type", "ne", 0))
    got = [[] for _ in qids]
    gotj = []
    cut = 3
    for i, b in enumerate(batches[:cut]):
        s.push(b.ts, b.key, b.value, b.type)
        if i < cut - 1:  # the last batch's rows stay unpolled across the snapshot
            for j, q in enumerate(qids):
                got[j].append(s.poll(q))
            gotj.append(s.poll_join(jid))
    st0 = s.stats()
    blob = s.snapshot()
    assert st0["state_groups"] > 0
    s.close()
    s = lm.Stream.restore(blob)
    try:
        st1 = s.stats()
        assert st1["batches"] == st0["batches"] and st1["watermark"] == st0["watermark"]
        assert st1["state_groups"] == st0["state_groups"]
        assert len(s.snapshot()) == len(blob)
        for j, q in enumerate(qids):
            got[j].append(s.poll(q))
        gotj.append(s.poll_join(jid))
        for i, b in enumerate(batches[cut:]):
            s.push(b.ts, b.key, b.value, b.type, eos=(cut + i == len(batches) - 1))
            for j, q in enumerate(qids):
                got[j].append(s.poll(q))
            gotj.append(s.poll_join(jid))
    finally:
        s.close()
    for j in range(len(qids)):
        _same(np.concatenate(got[j]), np.concatenate(ref_rows[j]), float_values, f"q{j}")
    _same_join(np.concatenate(gotj), np.concatenate(ref_join), float_values, "join")


def test_sharded_snapshot_restore():
    batches = _batches(61, n=20000, card=3000, lateness_jitter=40)
    kw = dict(value_type="int32", has_type=True, allowed_lateness_ms=25, key_fields=(8, 8))
    ref_rows, _ = _run(OracleShard(**kw), batches, QUERIES, join=False)
    sh = sharded.ShardedStream.open(3, devices=[0, 0, 0], key_mask=0xFF, **kw)
    qids = [sh.register_query(**q) for q in QUERIES]
    got = [[] for _ in qids]
    for b in batches[:4]:
        sh.push(b.ts, b.key, b.value, b.type)
        for j, q in enumerate(qids):
            got[j].append(sh.poll(q))
    blobs = sh.snapshot()
    order_by = dict(sh.order_by)
    sh.close()
    sh = sharded.ShardedStream.restore(blobs, devices=[0, 0, 0], key_mask=0xFF, order_by=order_by)
    try:
        for i, b in enumerate(batches[4:]):
            sh.push(b.ts, b.key, b.value, b.type, eos=(4 + i == len(batches) - 1))
            for j, q in enumerate(qids):
                got[j].append(sh.poll(q))
    finally:
        sh.close()
    for j in range(len(qids)):
        for b in range(len(batches)):
            _same(got[j][b], ref_rows[j][b], False, f"q{j} b{b}")
