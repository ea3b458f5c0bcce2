"""Continuous batching on the GPU: micro-batches of four streams (different
schemas, queries and sizes) submitted together to a server with three slots
run concurrently, and every stream's rows equal the rows of the same stream
processed alone (counts, integer sums, min and max exactly; float sums and
averages within engine_helpers.FLOAT_REL_TOL)."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import FLOAT_REL_TOL

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


def _same_rows(a, b, is_float, ctx):
    assert len(a) == len(b), ctx
    for f in ("window_start", "key", "count", "query_id"):
        np.testing.assert_array_equal(a[f], b[f], err_msg=ctx)
    if is_float:
        for f in ("min", "max"):
            np.testing.assert_array_equal(a[f].view(np.uint32), b[f].view(np.uint32), err_msg=ctx)
        for f in ("sum", "avg"):
            assert np.all(np.abs(a[f] - b[f]) <= FLOAT_REL_TOL * np.abs(b[f])), ctx
    else:
        for f in ("sum", "min", "max"):
            np.testing.assert_array_equal(a[f], b[f], err_msg=ctx)
        np.testing.assert_array_equal(a["avg"].view(np.uint64), b["avg"].view(np.uint64),
                                      err_msg=ctx)


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


def _mix(specs, budget):
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
    rows = [[s.poll(q) for q in range(len(sp["queries"]))] for s, sp in zip(streams, specs)]
    for s in streams:
        s.close()
    assert stats["completed"] == len(tickets)
    return rows, spans, stats


def test_results_alone_equal_results_in_the_mix():
    specs = _streams()
    alone = [_alone(sp)[0] for sp in specs]
    free, spans, stats = _mix(specs, 0)
    # then under a device memory budget just above what the mix ends up holding
    budget = int(1.1 * stats["held_bytes"])
    capped, _, cstats = _mix(specs, budget)
    exact = 0
    for k, sp in enumerate(specs):
        for q in range(len(sp["queries"])):
            assert len(alone[k][q]) > 0
            for got in (free[k][q], capped[k][q]):
                _same_rows(got, alone[k][q], sp["vt"] == "float32", f"stream {k} q{q}")
                exact += int(got.tobytes() == alone[k][q].tobytes())
    print(f"{exact} of {2 * sum(len(sp['queries']) for sp in specs)} row sets bit-identical; "
          f"server stats {stats}; with a {budget}-byte budget {cstats}")
    assert stats["max_concurrent"] >= 2
    overlap = any(a1 < b2 and a2 < b1 for (k1, a1, b1) in spans for (k2, a2, b2) in spans
                  if k1 != k2)
    assert overlap, "no two streams' micro-batches ran at the same time"
    assert cstats["peak_bytes"] <= budget
