"""Post-aggregation on the GPU against the oracle (Table III): LR2S-shaped
(GROUP BY packed (highway, direction, segment) fields of the key, HAVING
avg(speed) < 40, sliding 30 s / 10 s, int values), CM1-shaped (ORDER BY
SUM(cpu), tumbling and sliding, float values), HAVING and ORDER BY together,
and the ORDER BY size limit."""
import numpy as np
import pytest

from oracle import window_agg as wa
from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = (4, 1, 7, 20)  # highway, direction, segment, vehicle (bits)


def _lr_stream(seed, n_batches=4, n=30_000):
    rng = np.random.default_rng(seed)
    t = 0
    out = []
    for _ in range(n_batches):
        hw, dr = rng.integers(0, 10, n), rng.integers(0, 2, n)
        sg, vh = rng.integers(0, 100, n), rng.integers(0, 1 << 20, n)
        key = (hw | (dr << 4) | (sg << 5) | (vh << 12)).astype(np.uint32)
        ts = t + np.cumsum(rng.integers(0, 3, n)).astype(np.int64)
        t = int(ts[-1])
        val = rng.integers(0, 100, n).astype(np.int32)  # speeds
        out.append(synth.Batch(ts, key, val, None))
    return out


def _run_both(batches, is_float, q, key_fields=None):
    s = lm.Stream("float32" if is_float else "int32", key_fields=key_fields)
    qid = s.register_query(q["size"], q.get("slide", 0), q.get("col", "ts"), q.get("op", "none"),
                           q.get("value", 0), group_fields=q.get("fields", 0),
                           having=q.get("having"), order_by=q.get("order"))
    o = wa.WindowAggOracle(is_float, 0)
    oq = o.add_query(wa.COL_TS if q.get("col", "ts") == "ts" else wa.COL_VALUE,
                     {"none": wa.OP_NONE, "gt": wa.OP_GT}[q.get("op", "none")], 0,
                     float(q.get("value", 0)), q["size"], q.get("slide") or q["size"])
    mask = 0xFFFFFFFF
    if q.get("fields"):
        mask, shift = 0, 0
        for f, w in enumerate(key_fields):
            if (q["fields"] >> f) & 1:
                mask |= ((1 << w) - 1) << shift
            shift += w
    hv = q.get("having")
    o.set_post(oq, group_mask=mask,
               having=None if hv is None else (hv[0], {"lt": wa.OP_LT, "ge": wa.OP_GE}[hv[1]], hv[2]),
               order_by=q.get("order"))
    eng, orc = [], []
    for i, b in enumerate(batches):
        eos = i == len(batches) - 1
        s.push(b.ts, b.key, b.value, eos=eos)
        o.push(b.ts, b.key, b.value, None, eos=eos)
        eng.append(s.poll(qid))
        orc.append(o.take_rows(oq))
    s.close()
    o.close()
    return np.concatenate(eng), np.concatenate(orc)


def test_lr2s_group_by_fields_having_avg_below_40():
    q = dict(size=30_000, slide=10_000, fields=0b0111, having=("avg", "lt", 40.0))
    eng, orc = _run_both(_lr_stream(1), False, q, key_fields=FIELDS)
    assert len(orc) > 1000
    assert_rows_match(eng, orc, False)
    assert np.all(eng["avg"] < 40.0) and np.all(eng["key"] < (1 << 12))


@pytest.mark.parametrize("window", [dict(size=20_000), dict(size=60_000, slide=10_000)])
@pytest.mark.parametrize("desc", [True, False])
def test_cm1_order_by_sum(window, desc):
    s = synth.LargeFloatStream(seed=3, card=40, s=1.0)
    batches = [s.next_batch(n) for n in (40_000, 7, 55_555, 30_000)]
    q = dict(window, order=("sum", desc))
    eng, orc = _run_both(batches, True, q)
    assert len(orc) > 100
    assert_rows_match(eng, orc, True)


def test_having_and_order_by_together_with_filter():
    s = synth.LargeFloatStream(seed=4, card=500, s=1.2)
    batches = [s.next_batch(n) for n in (60_000, 60_000)]
    q = dict(size=10_000, slide=5_000, col="value", op="gt", value=0.5,
             having=("count", "ge", 3), order=("max", True))
    eng, orc = _run_both(batches, True, q)
    assert_rows_match(eng, orc, True)


def test_order_by_window_beyond_the_limit_is_rejected():
    n = lm.ORDER_MAX_ROWS + 100
    ts = np.zeros(n, np.int64)
    key = np.arange(n, dtype=np.uint32)
    val = np.ones(n, np.int32)
    s = lm.Stream("int32")
    s.register_query(1000, order_by=("sum", False))
    with pytest.raises(lm.LmsError) as ei:
        s.push(ts, key, val, eos=True)
    assert ei.value.status == lm.LMS_EINVAL
    s.close()
