"""TEST INFRASTRUCTURE ONLY: CPU oracle of the windowed equi-join of two streams.

Only tests, `__graft_entry__.smoke()` and bench.py's CPU legs may use it; the
engine's implementation (CUDA, in the library) shares no code with it.

The paper's LR1S / LR1T queries (Table III) join a windowed stream with a
stream on vehicle (`... FROM SegSpeedStr [range 30 (slide 5)] AS A,
SegSpeedStr AS L WHERE A.vehicle == L.vehicle`); Join is an operation of
Table II (base cost 0.9).  The paper leaves the semantics to Spark.  Reading
used here (the engine's): the two sides are the rows of one stream that pass
a left and a right predicate (for LR1, both sides are the whole stream); for
every window w (the event-time windows of the aggregation oracle, emitted when
the watermark passes them) the join result is the multiset L_w x R_w of pairs
(l, r) with l.key == r.key.  It is reported in factored form, one row per
(w, key) with both sides present:

    pairs       = |L_wk| * |R_wk|
    left_count  = |L_wk|,  right_count = |R_wk|
    left_sum    = sum of l.value over L_wk,  right_sum likewise
    (so that, e.g., the sum of l.value over all pairs is left_sum * right_count)

The per-side aggregates come from the aggregation oracle (window_agg, pinned
on its own); this module intersects them by (window start, key).  Pinned by
explicit enumeration of the pairs on tiny streams (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

from . import window_agg as wa

JOIN_ROW_DTYPE = np.dtype([("window_start", "<i8"), ("pairs", "<i8"), ("left_count", "<i8"),
                           ("right_count", "<i8"), ("left_sum", "<f8"), ("right_sum", "<f8"),
                           ("key", "<u4")])


class WindowJoinOracle:
    """left / right: (column, op, integer constant, float constant) predicates
    in the aggregation oracle's codes."""

    def __init__(self, value_is_float: bool, size_ms: int, slide_ms: int, left, right,
                 allowed_lateness_ms: int = 0):
        self.is_float = bool(value_is_float)
        self.o = wa.WindowAggOracle(value_is_float, allowed_lateness_ms)
        self.ql = self.o.add_query(left[0], left[1], left[2], left[3], size_ms, slide_ms)
        self.qr = self.o.add_query(right[0], right[1], right[2], right[3], size_ms, slide_ms)

    def push(self, ts, key, value, type_=None, eos=False, ts_floor=None) -> np.ndarray:
        """Feeds one micro-batch; returns the join rows of the windows it closed,
        ordered by (window start, key).  ts_floor: as WindowAggOracle.push."""
        self.o.push(ts, key, value, type_, eos=eos, ts_floor=ts_floor)
        lrows, rrows = self.o.take_rows(self.ql), self.o.take_rows(self.qr)
        right = {(int(r["window_start"]), int(r["key"])): r for r in rrows}
        out = []
        for l in lrows:  # already in (window start, key) order
            r = right.get((int(l["window_start"]), int(l["key"])))
            if r is None:
                continue
            sl = float(l["sum_f"]) if self.is_float else float(l["sum_i"])
            sr = float(r["sum_f"]) if self.is_float else float(r["sum_i"])
            out.append((int(l["window_start"]), int(l["count"]) * int(r["count"]), int(l["count"]),
                        int(r["count"]), sl, sr, int(l["key"])))
        return np.array(out, dtype=JOIN_ROW_DTYPE)

    def close(self):
        self.o.close()
