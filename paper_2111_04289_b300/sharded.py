"""Key-sharded streams over several GPUs (host logic; argument marshalling and
row merging only — every step of a shard's path runs in its own engine stream).

A window group (window, key) is built from the rows of its key alone, so the
key space splits over G streams, one per GPU: shard g owns the keys with
lms_shard_of(key, key_mask, G) == g (Table II's "Shuffling" operation, done on
the host before the copy to the device).  The one quantity every shard needs
from the whole micro-batch is its max event time, which advances the watermark
(Section II-A: event-time windows close on the max event time seen); each
shard is given it as a hint (lms_stream_set_batch_max_ts) and is pushed once
per global micro-batch, an empty shard included, so all shards close the same
windows.  The union of the shards' rows is the single stream's; merging
orders each window's rows by key (or by the ORDER BY aggregate, equal values
in key order), as one stream orders them.

ShardedStream drives G streams from one process (one per device).
DistShardedStream is one shard per rank of a torch.distributed group: each
rank brings the rows of its own input source; the rows are exchanged by
shard with one all-to-all per micro-batch and the max event time with one
all-reduce (the only collectives), then each rank pushes its shard.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import lmstream as lm

INT64_MIN = -(1 << 63)
INT64_MAX = (1 << 63) - 1
POST_FIELD = {"count": "count", "sum": "sum", "min": "min", "max": "max", "avg": "avg"}


def shard_of(key, key_mask: int, n_shards: int) -> np.ndarray:
    """lms_shard_of for every key of an array."""
    lib = lm.load()
    k = np.asarray(key, dtype=np.uint32).ravel()
    return np.fromiter((lib.lms_shard_of(int(x), int(key_mask) & 0xFFFFFFFF, int(n_shards))
                        for x in k), dtype=np.uint32, count=k.size)


def shard_split(ts, key, value, type_, n_shards: int, key_mask: int = 0xFFFFFFFF):
    """lms_shard_split of host columns: (list of G (ts, key, value, type) column
    views, in input order per shard; the batch's max ts or None if empty)."""
    lib = lm.load()
    ts = np.ascontiguousarray(ts, dtype=np.int64)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    value = np.ascontiguousarray(value)
    if value.dtype.itemsize != 4:
        raise ValueError("value column must be int32 or float32")
    n = int(ts.shape[0])
    b = lm.BatchC()
    b.n_rows = n
    b.ts, b.key, b.value = ts.ctypes.data, key.ctypes.data, value.ctypes.data
    tp = None
    if type_ is not None:
        type_ = np.ascontiguousarray(type_, dtype=np.uint8)
        b.type = type_.ctypes.data
        tp = np.empty(n, np.uint8)
    b.memory = lm.MEM_HOST
    o_ts = np.empty(n, np.int64)
    o_key = np.empty(n, np.uint32)
    o_val = np.empty(n, value.dtype)
    offs = np.zeros(n_shards + 1, np.int64)
    mx = ctypes.c_int64()
    st = lib.lms_shard_split(ctypes.byref(b), int(key_mask) & 0xFFFFFFFF, int(n_shards),
                             o_ts.ctypes.data, o_key.ctypes.data, o_val.ctypes.data,
                             None if tp is None else tp.ctypes.data, offs.ctypes.data,
                             ctypes.byref(mx))
    if st != lm.LMS_OK:
        raise lm.LmsError(st, "lms_shard_split")
    parts = []
    for g in range(n_shards):
        a, e = int(offs[g]), int(offs[g + 1])
        parts.append((o_ts[a:e], o_key[a:e], o_val[a:e], None if tp is None else tp[a:e]))
    return parts, (None if n == 0 else int(mx.value))


def _order_code(x: np.ndarray, desc: bool) -> np.ndarray:
    """Order-preserving uint64 code of doubles (both zeros equal), the order the
    engine's ORDER BY sorts by."""
    x = np.where(x == 0.0, 0.0, x).astype(np.float64)
    u = x.view(np.uint64)
    code = np.where(u >> np.uint64(63) != 0, ~u, u | np.uint64(1 << 63))
    return ~code if desc else code


def merge_rows(parts: Sequence[np.ndarray], order_by=None, is_float: bool = False) -> np.ndarray:
    """Merges the shards' rows of a batch: by (window_start, key), or with
    order_by = (agg, descending) by (window_start, aggregate, key)."""
    parts = [p for p in parts if len(p)]
    if not parts:
        return np.zeros(0, lm.ROW_DTYPE_FLOAT if is_float else lm.ROW_DTYPE_INT)
    rows = np.concatenate(parts)
    if order_by is None:
        idx = np.lexsort((rows["key"], rows["window_start"]))
    else:
        agg, desc = order_by
        v = rows[POST_FIELD[agg]].astype(np.float64)
        idx = np.lexsort((rows["key"], _order_code(v, bool(desc)), rows["window_start"]))
    return rows[idx]


def merge_join_rows(parts: Sequence[np.ndarray]) -> np.ndarray:
    parts = [p for p in parts if len(p)]
    if not parts:
        return None
    rows = np.concatenate(parts)
    return rows[np.lexsort((rows["key"], rows["window_start"]))]


class ShardedStream:
    """G engine streams (one per device) that together run one stream's queries,
    each owning the keys lms_shard_of assigns it."""

    def __init__(self, shards: Sequence, key_mask: int = 0xFFFFFFFF,
                 origin_ts: Optional[int] = None):
        self.shards = list(shards)
        self.n = len(self.shards)
        if self.n < 1:
            raise ValueError("need at least one shard")
        self.key_mask = int(key_mask) & 0xFFFFFFFF
        self.origin_ts = origin_ts
        self._origin_done = False
        self.order_by = {}
        self.is_float = getattr(self.shards[0], "is_float", False)
        if origin_ts is not None:
            self._set_origin(int(origin_ts))

    @classmethod
    def open(cls, n_shards: int, devices: Optional[Sequence[int]] = None,
             key_mask: int = 0xFFFFFFFF, origin_ts: Optional[int] = None, **stream_kwargs):
        """n_shards engine streams on `devices` (default: shard g on device g)."""
        devices = list(range(n_shards)) if devices is None else list(devices)
        if len(devices) != n_shards:
            raise ValueError("one device per shard")
        shards = [lm.Stream(device=d, **stream_kwargs) for d in devices]
        return cls(shards, key_mask=key_mask, origin_ts=origin_ts)

    def _set_origin(self, origin: int):
        for s in self.shards:
            s.set_origin(origin)
        self.origin_ts = origin
        self._origin_done = True

    def register_query(self, *args, **kw) -> int:
        ids = {s.register_query(*args, **kw) for s in self.shards}
        assert len(ids) == 1
        qid = ids.pop()
        self.order_by[qid] = kw.get("order_by")
        return qid

    def register_join(self, *args, **kw) -> int:
        ids = {s.register_join(*args, **kw) for s in self.shards}
        assert len(ids) == 1
        return ids.pop()

    def push(self, ts, key, value, type_=None, eos: bool = False) -> int:
        """One global micro-batch (host columns): split by key, every shard
        pushed with the batch's max event time as its watermark hint."""
        parts, mx = shard_split(ts, key, value, type_, self.n, self.key_mask)
        if not self._origin_done and mx is not None:
            # the single stream's automatic origin: the first row of the first batch
            self._set_origin(int(np.asarray(ts)[0]))
        for s, (t, k, v, y) in zip(self.shards, parts):
            if mx is not None:
                s.set_batch_max_ts(mx)
            s.push(t, k, v, y, eos=eos)
        return int(np.asarray(ts).shape[0])

    def poll(self, qid: int) -> np.ndarray:
        return merge_rows([s.poll(qid) for s in self.shards], self.order_by.get(qid),
                          self.is_float)

    def poll_join(self, jid: int) -> np.ndarray:
        parts = [s.poll_join(jid) for s in self.shards]
        m = merge_join_rows(parts)
        return parts[0][:0] if m is None else m

    def snapshot(self) -> list:
        return [s.snapshot() for s in self.shards]

    @classmethod
    def restore(cls, blobs: Sequence[bytes], devices: Optional[Sequence[int]] = None,
                key_mask: int = 0xFFFFFFFF, order_by=None):
        devices = [-1] * len(blobs) if devices is None else list(devices)
        shards = [lm.Stream.restore(b, d) for b, d in zip(blobs, devices)]
        self = cls(shards, key_mask=key_mask)
        self._origin_done = True  # a restored stream keeps its origin
        self.order_by = dict(order_by or {})
        return self

    def close(self):
        for s in self.shards:
            s.close()


class DistShardedStream:
    """One key shard per rank of a torch.distributed group.  `stream` is this
    rank's stream (an engine Stream on its own GPU); each rank pushes the rows of
    its own input source, and the rows are exchanged so that every rank gets
    the rows of the keys it owns."""

    def __init__(self, stream, group=None, key_mask: int = 0xFFFFFFFF,
                 origin_ts: Optional[int] = None, comm_device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.s = stream
        self.group = group
        self.rank = dist.get_rank(group)
        self.n = dist.get_world_size(group)
        self.key_mask = int(key_mask) & 0xFFFFFFFF
        if comm_device is None:
            comm_device = ("cuda" if dist.get_backend(group) == "nccl" else "cpu")
        self.dev = torch.device(comm_device)
        self._origin_done = False
        self.order_by = {}
        self.is_float = getattr(stream, "is_float", False)
        if origin_ts is not None:
            self.s.set_origin(int(origin_ts))
            self._origin_done = True

    def register_query(self, *args, **kw) -> int:
        qid = self.s.register_query(*args, **kw)
        self.order_by[qid] = kw.get("order_by")
        return qid

    def register_join(self, *args, **kw) -> int:
        return self.s.register_join(*args, **kw)

    def _all_reduce(self, x: int, op) -> int:
        t = self.torch.tensor([x], dtype=self.torch.int64, device=self.dev)
        self.dist.all_reduce(t, op=op, group=self.group)
        return int(t.item())

    def _exchange(self, col: np.ndarray, send: list, recv: list) -> np.ndarray:
        t = self.torch.from_numpy(np.ascontiguousarray(col)).to(self.dev)
        out = self.torch.empty(int(sum(recv)), dtype=t.dtype, device=self.dev)
        self.dist.all_to_all_single(out, t, recv, send, group=self.group)
        return out.cpu().numpy()

    def push(self, ts, key, value, type_=None, eos: bool = False) -> int:
        """This rank's source rows of one global micro-batch; returns the rows
        this rank's shard received."""
        dist = self.dist
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        parts, mx = shard_split(ts, key, value, type_, self.n, self.key_mask)
        send = [int(p[0].shape[0]) for p in parts]
        cnt = self.torch.tensor(send, dtype=self.torch.int64, device=self.dev)
        got = self.torch.empty(self.n, dtype=self.torch.int64, device=self.dev)
        dist.all_to_all_single(got, cnt, group=self.group)
        recv = [int(x) for x in got.cpu().tolist()]
        vdt = np.asarray(value).dtype

        def col(i):
            return np.concatenate([p[i] for p in parts]) if parts else np.zeros(0)
        r_ts = self._exchange(col(0), send, recv)
        r_key = self._exchange(col(1).view(np.int32), send, recv).view(np.uint32)
        r_val = self._exchange(col(2).view(np.int32), send, recv).view(vdt)
        r_typ = None
        if type_ is not None:
            r_typ = self._exchange(col(3), send, recv)
        # the batch's max event time over every source, and (first batch) the
        # origin: the earliest first row of the sources' first batches
        gmx = self._all_reduce(INT64_MIN if mx is None else mx, dist.ReduceOp.MAX)
        if not self._origin_done:
            first = self._all_reduce(int(ts[0]) if ts.shape[0] else INT64_MAX,
                                     dist.ReduceOp.MIN)
            if first != INT64_MAX:
                self.s.set_origin(first)
                self._origin_done = True
        if gmx != INT64_MIN:
            self.s.set_batch_max_ts(gmx)
        self.s.push(r_ts, r_key, r_val, r_typ, eos=eos)
        return int(r_ts.shape[0])

    def poll(self, qid: int) -> np.ndarray:
        """This rank's shard rows."""
        return self.s.poll(qid)

    def gather(self, qid: int, dst: int = 0):
        """The merged rows of every shard on rank dst (None elsewhere)."""
        mine = self.s.poll(qid)
        out = [None] * self.n if self.rank == dst else None
        self.dist.gather_object(mine, out, dst=dst, group=self.group)
        if self.rank != dst:
            return None
        return merge_rows(out, self.order_by.get(qid), self.is_float)
