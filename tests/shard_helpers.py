"""An oracle-backed stand-in for one shard's engine stream (CPU, tests only):
the same methods as lmstream.Stream that the sharded host logic calls, with
rows converted to the engine's row layout, so that the host logic (split,
watermark agreement, exchange, merge) is tested without a GPU."""
from __future__ import annotations

import numpy as np

from oracle import join as oj
from oracle import window_agg as wa
from paper_2111_04289_b300 import lmstream as lm

COL = {"ts": wa.COL_TS, "key": wa.COL_KEY, "value": wa.COL_VALUE, "type": wa.COL_TYPE}
OP = {"none": wa.OP_NONE, "eq": wa.OP_EQ, "ne": wa.OP_NE, "lt": wa.OP_LT, "le": wa.OP_LE,
      "gt": wa.OP_GT, "ge": wa.OP_GE}


def group_mask(key_fields, group_fields: int) -> int:
    if not group_fields:
        return 0xFFFFFFFF
    m, shift = 0, 0
    for f, w in enumerate(key_fields):
        if (group_fields >> f) & 1:
            m |= ((1 << w) - 1) << shift
        shift += w
    return m


def to_engine_rows(r: np.ndarray, is_float: bool) -> np.ndarray:
    out = np.zeros(len(r), lm.ROW_DTYPE_FLOAT if is_float else lm.ROW_DTYPE_INT)
    out["window_start"] = r["window_start"]
    out["count"] = r["count"]
    out["avg"] = r["avg"]
    out["key"] = r["key"]
    if is_float:
        out["sum"], out["min"], out["max"] = r["sum_f"], r["min_f"], r["max_f"]
    else:
        out["sum"], out["min"], out["max"] = r["sum_i"], r["min_i"], r["max_i"]
    return out


class OracleShard:
    def __init__(self, value_type="int32", allowed_lateness_ms=0, key_fields=(), **_engine_only):
        self.is_float = value_type == "float32"
        self.lateness = allowed_lateness_ms
        self.key_fields = tuple(key_fields)
        self.o = wa.WindowAggOracle(self.is_float, allowed_lateness_ms)
        self.joins = []
        self.floor = None
        self.pending = {}
        self.join_pending = {}

    def register_query(self, size_ms, slide_ms=0, filter_col="ts", filter_op="none",
                       filter_value=0, agg_mask=lm.AGG_ALL, group_fields=0, having=None,
                       order_by=None):
        fv = filter_value
        q = self.o.add_query(COL[filter_col], OP[filter_op], 0 if isinstance(fv, float) else int(fv),
                             float(fv), size_ms, slide_ms or size_ms)
        h = None if having is None else (having[0], OP[having[1]], having[2])
        self.o.set_post(q, group_mask(self.key_fields, group_fields), h, order_by)
        self.pending[q] = []
        return q

    def register_join(self, size_ms, slide_ms=0, left=("ts", "none", 0), right=("ts", "none", 0)):
        def pred(p):
            c, op, v = p
            return (COL[c], OP[op], 0 if isinstance(v, float) else int(v), float(v))
        j = oj.WindowJoinOracle(self.is_float, size_ms, slide_ms or size_ms, pred(left),
                                pred(right), self.lateness)
        self.joins.append(j)
        self.join_pending[len(self.joins) - 1] = []
        return len(self.joins) - 1

    def set_origin(self, origin_ts):
        pass  # the oracle's windows are absolute

    def set_batch_max_ts(self, ts):
        self.floor = int(ts)

    def push(self, ts, key, value, type_=None, eos=False):
        f, self.floor = self.floor, None
        self.o.push(ts, key, value, type_, eos=eos, ts_floor=f)
        for q in self.pending:
            self.pending[q].append(to_engine_rows(self.o.take_rows(q), self.is_float))
        for i, j in enumerate(self.joins):
            self.join_pending[i].append(j.push(ts, key, value, type_, eos=eos, ts_floor=f))
        return len(ts)

    def poll(self, qid):
        p = self.pending[qid]
        self.pending[qid] = []
        return (np.concatenate(p) if p else
                np.zeros(0, lm.ROW_DTYPE_FLOAT if self.is_float else lm.ROW_DTYPE_INT))

    def poll_join(self, jid):
        p = self.join_pending[jid]
        self.join_pending[jid] = []
        return np.concatenate(p) if p else np.zeros(0, oj.JOIN_ROW_DTYPE)
