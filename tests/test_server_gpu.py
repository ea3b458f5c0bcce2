"""Continuous batching on the GPU: micro-batches of four streams (different
schemas, queries and sizes) submitted together to a server with three slots
run concurrently, and every stream's rows equal the rows of the same stream
processed alone (counts, integer sums, min and max exactly; float sums and
averages within engine_helpers.FLOAT_REL_TOL)."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _streams():
    lf = synth.LargeFloatStream(seed=71)
    ti = synth.TinyIntStream(seed=72, card=1024)
    lf2 = synth.LargeFloatStream(seed=73, card=20_000)
    ti2 = synth.TinyIntStream(seed=74, card=50)
    sizes = [2 ** 14, 3 * 2 ** 15, 2 ** 17 + 77, 2 ** 16, 5_000, 2 ** 18]
    return [
        dict(vt="float32", has_type=False, batches=[lf.next_batch(n) for n in sizes],
             queries=[(60_000, 5_000, "value", "gt", 0.5)]),
        dict(vt="int32", has_type=True, batches=[ti.next_batch(n) for n in sizes[::-1]],
             queries=[(10_000, 0, "type", "eq", 0)]),
        dict(vt="float32", has_type=False, batches=[lf2.next_batch(n) for n in sizes[1:]],
             queries=[(30_000, 1_000, "value", "gt", 1.0), (10_000, 0, "ts", "none", 0)]),
        dict(vt="int32", has_type=True, batches=[ti2.next_batch(n) for n in sizes[:4]],
             queries=[(3_000, 1_000, "key", "lt", 25)]),
    ]


def _open(spec):
    s = lm.Stream(spec["vt"], has_type=spec["has_type"])
    for (size, slide, col, op, v) in spec["queries"]:
        s.register_query(size, slide, col, op, v)
    return s


def _alone(spec):
    s = _open(spec)
    out = [[] for _ in spec["queries"]]
    for i, b in enumerate(spec["batches"]):
        s.push(b.ts, b.key, b.value, b.type, eos=i == len(spec["batches"]) - 1)
        for q in range(len(spec["queries"])):
            out[q].append(s.poll(q))
    dev = s.stats()["device_bytes"]
    s.close()
    return [np.concatenate(r) for r in out], dev


@pytest.mark.parametrize("budget_factor", [0.0, 1.3])
def test_results_alone_equal_results_in_the_mix(budget_factor):
    specs = _streams()
    alone, devs = zip(*[_alone(sp) for sp in specs])
    budget = int(budget_factor * sum(devs))
    sv = lm.Server(slots=3, memory_budget_bytes=budget)
    streams = [_open(sp) for sp in specs]
    tickets = []
    rounds = max(len(sp["batches"]) for sp in specs)
    for i in range(rounds):  # interleave the streams' batches
        for k, sp in enumerate(specs):
            if i < len(sp["batches"]):
                b = sp["batches"][i]
                t = sv.submit(streams[k], b.ts, b.key, b.value, b.type,
                              eos=i == len(sp["batches"]) - 1)
                tickets.append((k, t))
    spans = []
    for k, t in tickets:
        st, a, b = sv.wait(t)
        assert st == lm.LMS_OK
        spans.append((k, a, b))
    stats = sv.stats()
    sv.close()
    exact = 0
    for k, sp in enumerate(specs):
        for q in range(len(sp["queries"])):
            got = streams[k].poll(q)
            assert_rows_match(got, alone[k][q], sp["vt"] == "float32", ctx=f"stream {k} q{q}")
            exact += int(got.tobytes() == alone[k][q].tobytes())
        streams[k].close()
    print(f"{exact} of {sum(len(sp['queries']) for sp in specs)} row sets bit-identical; "
          f"server stats {stats}")
    assert stats["completed"] == len(tickets)
    assert stats["max_concurrent"] >= 2
    overlap = any(a1 < b2 and a2 < b1 for (k1, a1, b1) in spans for (k2, a2, b2) in spans
                  if k1 != k2)
    assert overlap, "no two streams' micro-batches ran at the same time"
    if budget:
        assert stats["peak_bytes"] <= budget
