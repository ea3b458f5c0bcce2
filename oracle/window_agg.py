"""TEST INFRASTRUCTURE ONLY: Python loader for the C++ windowed-aggregation oracle.

The semantics are written out at the top of `window_agg_oracle.cpp` (event-time
tumbling / sliding windows, group-by count/sum/min/max/avg, watermark emission).
The paper (LMStream, Table III) states its queries as SQL over windows but
leaves window semantics to Spark; the oracle fixes them as described there.

Only tests, `__graft_entry__.smoke()` and `bench.py --impl reference` /
the `cpu_baseline` leg may use this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "window_agg_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libwindow_agg_oracle.so")
_lock = threading.Lock()
_lib = None

# Column / operator codes of the oracle (its own numbering, mirrored by name in
# the engine's public header because both follow the same query description).
COL_TS, COL_KEY, COL_VALUE, COL_TYPE = 0, 1, 2, 3
OP_NONE, OP_EQ, OP_NE, OP_LT, OP_LE, OP_GT, OP_GE = 0, 1, 2, 3, 4, 5, 6
# Aggregates a HAVING or ORDER BY refers to.
AGGS = {"count": 1, "sum": 2, "min": 3, "max": 4, "avg": 5}

ROW_DTYPE = np.dtype(
    [
        ("window_start", "<i8"),
        ("window_end", "<i8"),
        ("count", "<i8"),
        ("sum_i", "<i8"),
        ("sum_f", "<f8"),
        ("avg", "<f8"),
        ("min_i", "<i4"),
        ("max_i", "<i4"),
        ("min_f", "<f4"),
        ("max_f", "<f4"),
        ("key", "<u4"),
        ("pad", "<u4"),
    ]
)


def build(force: bool = False) -> str:
    """Compiles the oracle with g++ (host only) and returns the .so path."""
    with _lock:
        if (
            not force
            and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
        ):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_open.restype = ctypes.c_void_p
        lib.oracle_open.argtypes = [ctypes.c_int, ctypes.c_int64]
        lib.oracle_close.argtypes = [ctypes.c_void_p]
        lib.oracle_add_query.restype = ctypes.c_int
        lib.oracle_add_query.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
            ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
        ]
        lib.oracle_push.restype = ctypes.c_int
        lib.oracle_push.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
        ]
        lib.oracle_push_floor.restype = ctypes.c_int
        lib.oracle_push_floor.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
        ]
        lib.oracle_pending_rows.restype = ctypes.c_int64
        lib.oracle_pending_rows.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_take_rows.restype = ctypes.c_int64
        lib.oracle_take_rows.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
        ]
        lib.oracle_late_rows.restype = ctypes.c_int64
        lib.oracle_late_rows.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_open_groups.restype = ctypes.c_int64
        lib.oracle_open_groups.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_set_post.restype = ctypes.c_int
        lib.oracle_set_post.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_int,
        ]
        lib.oracle_row_size.restype = ctypes.c_int64
        assert lib.oracle_row_size() == ROW_DTYPE.itemsize
        _lib = lib
    return _lib


class WindowAggOracle:
    """Per-event oracle stream: add queries, push micro-batches, take rows."""

    def __init__(self, value_is_float: bool, allowed_lateness_ms: int = 0):
        self._lib = _load()
        self.value_is_float = bool(value_is_float)
        self._h = self._lib.oracle_open(int(self.value_is_float), int(allowed_lateness_ms))

    def close(self):
        if self._h:
            self._lib.oracle_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_query(self, filter_col=COL_TS, filter_op=OP_NONE, filter_i=0,
                  filter_f=0.0, size_ms=1000, slide_ms=None) -> int:
        slide = size_ms if not slide_ms else slide_ms
        q = self._lib.oracle_add_query(
            self._h, int(filter_col), int(filter_op), int(filter_i),
            float(filter_f), int(size_ms), int(slide),
        )
        if q < 0:
            raise ValueError("invalid window: size must be a positive multiple of slide")
        return q

    def set_post(self, qid: int, group_mask: int = 0xFFFFFFFF, having=None, order_by=None):
        """Post-aggregation of query qid: group by key & group_mask; having =
        (agg, op, value) keeps rows with (double)agg OP value; order_by =
        (agg, descending) sorts each window's rows by the aggregate (ties in key
        order).  agg: one of AGGS."""
        ha, ho, hv = (0, OP_NONE, 0.0) if having is None else (AGGS[having[0]], having[1],
                                                               float(having[2]))
        oa, od = (0, 0) if order_by is None else (AGGS[order_by[0]], int(bool(order_by[1])))
        if self._lib.oracle_set_post(self._h, int(qid), int(group_mask) & 0xFFFFFFFF, ha, int(ho),
                                     hv, oa, od) != 0:
            raise ValueError("bad post-aggregation")

    def push(self, ts, key, value, type_=None, eos: bool = False, ts_floor=None):
        """One micro-batch; ts_floor: a lower bound of the batch's max event
        time (the whole micro-batch's, when this stream holds one key shard)."""
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        key = np.ascontiguousarray(key, dtype=np.uint32)
        value = np.ascontiguousarray(
            value, dtype=np.float32 if self.value_is_float else np.int32
        )
        n = ts.shape[0]
        assert key.shape[0] == n and value.shape[0] == n
        tp = None
        if type_ is not None:
            type_ = np.ascontiguousarray(type_, dtype=np.uint8)
            assert type_.shape[0] == n
            tp = type_.ctypes.data
        self._lib.oracle_push_floor(
            self._h, n, ts.ctypes.data, key.ctypes.data, value.ctypes.data, tp,
            int(bool(eos)), -(1 << 63) if ts_floor is None else int(ts_floor),
        )

    def take_rows(self, qid: int) -> np.ndarray:
        m = self._lib.oracle_pending_rows(self._h, qid)
        out = np.zeros(m, dtype=ROW_DTYPE)
        if m:
            got = self._lib.oracle_take_rows(self._h, qid, out.ctypes.data, m)
            assert got == m
        return out

    def late_rows(self, qid: int) -> int:
        return int(self._lib.oracle_late_rows(self._h, qid))

    def open_groups(self, qid: int) -> int:
        return int(self._lib.oracle_open_groups(self._h, qid))
