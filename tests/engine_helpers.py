"""Helpers shared by the GPU parity tests: run the same seeded micro-batches
through the CUDA engine (via the C ABI binding) and through the CPU oracle, and
compare their rows field by field."""
from __future__ import annotations

import numpy as np

from oracle import window_agg as wa
from paper_2111_04289_b300 import lmstream as lm

# Tolerance for floating sums/averages: FP64 accumulation in a different order
# than the oracle's sequential sum; values are positive in every workload, so
# the relative error is bounded by ~n*2^-53 << 1e-9.
FLOAT_REL_TOL = 1e-9

ORACLE_COL = {"ts": wa.COL_TS, "key": wa.COL_KEY, "value": wa.COL_VALUE, "type": wa.COL_TYPE}
ORACLE_OP = {"none": wa.OP_NONE, "eq": wa.OP_EQ, "ne": wa.OP_NE, "lt": wa.OP_LT,
             "le": wa.OP_LE, "gt": wa.OP_GT, "ge": wa.OP_GE}


def run_oracle(batches, queries, is_float, lateness=0, eos=True):
    o = wa.WindowAggOracle(is_float, lateness)
    qids = []
    for q in queries:
        fv = q.get("value", 0)
        qids.append(o.add_query(ORACLE_COL[q.get("col", "ts")], ORACLE_OP[q.get("op", "none")],
                                0 if isinstance(fv, float) else int(fv), float(fv),
                                q["size"], q.get("slide") or q["size"]))
    out = [[] for _ in queries]
    for i, b in enumerate(batches):
        o.push(b.ts, b.key, b.value, b.type, eos=(eos and i == len(batches) - 1))
        for j, qid in enumerate(qids):
            out[j].append(o.take_rows(qid))
    late = [o.late_rows(q) for q in qids]
    return [np.concatenate(r) if r else np.zeros(0, wa.ROW_DTYPE) for r in out], late


def run_engine(batches, queries, is_float, lateness=0, eos=True, has_type=None, device_input=False,
               torch=None, **kw):
    if has_type is None:
        has_type = batches[0].type is not None if batches else False
    s = lm.Stream("float32" if is_float else "int32", has_type=has_type,
                  allowed_lateness_ms=lateness, **kw)
    qids = []
    for q in queries:
        qids.append(s.register_query(q["size"], q.get("slide", 0), q.get("col", "ts"),
                                     q.get("op", "none"), q.get("value", 0)))
    out = [[] for _ in queries]
    for i, b in enumerate(batches):
        cols = [b.ts, b.key, b.value, b.type if has_type else None]
        if device_input:
            cols = [None if c is None else torch.from_numpy(np.ascontiguousarray(c)).cuda()
                    for c in cols]
        s.push(cols[0], cols[1], cols[2], cols[3], eos=(eos and i == len(batches) - 1))
        for j, qid in enumerate(qids):
            out[j].append(s.poll(qid))
    st = s.stats()
    s.close()
    return [np.concatenate(r) if r else np.zeros(0, s.row_dtype) for r in out], st


def assert_rows_match(eng, orc, is_float, size=None, ctx=""):
    assert len(eng) == len(orc), f"{ctx}: {len(eng)} engine rows vs {len(orc)} oracle rows"
    if len(eng) == 0:
        return
    np.testing.assert_array_equal(eng["window_start"], orc["window_start"], err_msg=ctx)
    np.testing.assert_array_equal(eng["key"], orc["key"], err_msg=ctx)
    np.testing.assert_array_equal(eng["count"], orc["count"], err_msg=ctx)
    if is_float:
        # min/max compared bitwise (totalOrder: -0.0 != +0.0)
        np.testing.assert_array_equal(eng["min"].view(np.uint32), orc["min_f"].view(np.uint32),
                                      err_msg=ctx)
        np.testing.assert_array_equal(eng["max"].view(np.uint32), orc["max_f"].view(np.uint32),
                                      err_msg=ctx)
        exp = orc["sum_f"]
        err = np.abs(eng["sum"] - exp)
        assert np.all(err <= FLOAT_REL_TOL * np.abs(exp) + 1e-300), f"{ctx}: sum max rel err"
        exp = orc["avg"]
        err = np.abs(eng["avg"] - exp)
        assert np.all(err <= FLOAT_REL_TOL * np.abs(exp) + 1e-300), f"{ctx}: avg"
    else:
        np.testing.assert_array_equal(eng["sum"], orc["sum_i"], err_msg=ctx)
        np.testing.assert_array_equal(eng["min"], orc["min_i"], err_msg=ctx)
        np.testing.assert_array_equal(eng["max"], orc["max_i"], err_msg=ctx)
        np.testing.assert_array_equal(eng["avg"].view(np.uint64), orc["avg"].view(np.uint64),
                                      err_msg=ctx)
