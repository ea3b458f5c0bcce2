"""Windowed equi-join on the GPU against the join oracle (LR1S / LR1T of
Table III): two sides told apart by the type column (tumbling 10 s, sliding
30 s / 5 s), a self-join, float and int values, several batches, and the
query-slot limit."""
import numpy as np
import pytest

from oracle import join as oj
from oracle import window_agg as wa
from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COL = {"ts": wa.COL_TS, "type": wa.COL_TYPE, "value": wa.COL_VALUE}
OP = {"none": wa.OP_NONE, "eq": wa.OP_EQ, "gt": wa.OP_GT}


def _two_streams(seed, sizes, card=100_000, s=1.1):
    g = synth.LargeFloatStream(seed=seed, card=card, s=s, with_type=True)
    out = []
    for n in sizes:
        b = g.next_batch(n)
        b.type = (b.type % 2).astype(np.uint8)  # side 0 / side 1
        out.append(b)
    return out


def _run(batches, is_float, size, slide, left, right):
    s = lm.Stream("float32" if is_float else "int32", has_type=True)
    jid = s.register_join(size, slide, left=left, right=right)
    o = oj.WindowJoinOracle(is_float, size, slide or size,
                            (COL[left[0]], OP[left[1]], int(left[2]), float(left[2])),
                            (COL[right[0]], OP[right[1]], int(right[2]), float(right[2])))
    eng, orc = [], []
    for i, b in enumerate(batches):
        val = b.value if is_float else (b.value * 100).astype(np.int32)
        eos = i == len(batches) - 1
        s.push(b.ts, b.key, val, b.type, eos=eos)
        eng.append(s.poll_join(jid))
        orc.append(o.push(b.ts, b.key, val, b.type, eos=eos))
    s.close()
    o.close()
    return np.concatenate(eng), np.concatenate(orc)


def _match(e, o, is_float):
    assert len(e) == len(o) > 0
    for f in ("window_start", "key", "pairs", "left_count", "right_count"):
        np.testing.assert_array_equal(e[f], o[f], err_msg=f)
    for f in ("left_sum", "right_sum"):
        if is_float:
            assert np.all(np.abs(e[f] - o[f]) <= 1e-9 * np.abs(o[f]) + 1e-300), f
        else:
            np.testing.assert_array_equal(e[f].astype(np.float64), o[f], err_msg=f)


@pytest.mark.parametrize("is_float", [True, False])
@pytest.mark.parametrize("size,slide", [(10_000, 0), (30_000, 5_000)])
def test_two_sided_join_equals_the_oracle(is_float, size, slide):
    batches = _two_streams(21, [50_000, 3, 70_000, 40_000])
    e, o = _run(batches, is_float, size, slide, ("type", "eq", 0), ("type", "eq", 1))
    _match(e, o, is_float)
    assert np.array_equal(e["pairs"], e["left_count"] * e["right_count"])


def test_self_join_of_a_filtered_side():
    batches = _two_streams(22, [30_000, 30_000], card=5_000, s=1.3)
    e, o = _run(batches, True, 5_000, 1_000, ("value", "gt", 1.0), ("ts", "none", 0))
    _match(e, o, True)


def test_join_takes_two_query_slots():
    s = lm.Stream("int32", has_type=True)
    for _ in range(7):
        s.register_query(1000)
    with pytest.raises(lm.LmsError) as ei:
        s.register_join(1000)
    assert ei.value.status == lm.LMS_EINVAL
    s.close()
